/*
 * dqmc.h - C ABI of the GB300 library for the data-parallel hot path of
 * real-space variational Monte Carlo with a DeepQMC-style neural-network
 * wave function (Schätzle, Szabó, Mezera, Hermann, Noé: "DeepQMC: an
 * open-source software suite for variational optimization of deep-learning
 * molecular wave functions", 2023).
 *
 * The ansatz instance (Sec. 3 of the paper):
 *   - graph over electrons and nuclei; edge features are a Gaussian expansion
 *     of the inter-particle distance (n_rbf Gaussians, centres q*rc/(n_rbf-1),
 *     width rc/(n_rbf-1)), reused in every layer (Eqs. 15-16, first case);
 *   - electron embeddings start from a spin-only embedding (Eq. 13, first
 *     case) and are updated n_layers times by graph convolutions (Eq. 17)
 *     over same-spin, opposite-spin and electron-nucleus edges, each sum
 *     normalised by its number of edges, with the concatenating residual
 *     update f <- f + tanh(W_g [m_par; m_anti; m_nuc] + b_g) (Eq. 18);
 *     edge filters w(e) = W2 tanh(W1 e + b1) + b2; node map z_j = W_h f_j;
 *     nucleus nodes carry a learnt vector Y_I per layer (Eq. 14);
 *   - orbitals: linear head on f^L (Eq. 19) times isotropic Slater envelopes
 *     sum_I omega exp(-zeta |r - R_I|) (Eq. 20);
 *   - psi = sum_p c_p det A^{up,p} det A^{down,p} (Eq. 21) in the log domain
 *     with log-sum-exp over p (Eqs. 27-28), times exp(J) with the learnable
 *     Jastrow J = w_J2 . tanh(W_J1 sum_i f_i^L + b_J1) (Eq. 24) and the
 *     electron cusp gamma = -sum_{i<j} alpha c_ij / (1 + alpha r_ij),
 *     c = 1/4 (same spin) or 1/2 (opposite spin) (Eq. 25).
 *
 * Electrons are spin-sorted: the first n_up are spin up (Sec. 2.2).
 * Units: bohr and hartree.
 *
 * Flat parameter vector (same dtype as the handle's arithmetic, see below),
 * matrices [out][in] row-major, in this order:
 *   E_spin[2][D], or with el_init W_e1[D][3 n_nuc], b_e1[D], W_e2[D][D], b_e2[D];
 *   per layer l < n_layers:
 *     W_h[D][D];
 *     for the edge types same-spin, opposite-spin, electron-nucleus:
 *       [U[n_rbf][n_rbf], c[n_rbf]: only with edge_update and l >= 1],
 *       W1[D][n_rbf], b1[D], W2[D][D], b2[D];
 *     Y[n_nuc][D]; W_g[D][3D], b_g[D];
 *   for spin up then spin down (n_c orbitals per determinant: n_s, the
 *   electrons of that spin, or N with full_det):
 *     W_o[K n_c][D], b_o[K n_c], omega[K n_c][n_nuc], zeta[K n_c][n_nuc]
 *     (orbital row p*n_c + k is orbital k of determinant p);
 *   c[K]; W_J1[D][D], b_J1[D], w_J2[D].
 *
 * Memory and dtypes.  Every array argument of a compute call is DEVICE memory
 * owned by the caller, on the device that was current at dq_create.  The
 * handle's precision fixes the dtype of params, r, logabs, e_loc, weights and
 * grad_out: double for DQ_FP64, float for DQ_FP32 and DQ_BF16_MIXED.  sign is
 * int8.  Sums written to double* arguments are FP64 in every mode.
 *
 * Workspace.  Compute calls allocate nothing: the caller passes a device
 * workspace of at least dq_workspace_size() bytes (256-byte aligned).
 * Walkers are processed in chunks of at most dq_max_chunk() walkers, so the
 * workspace does not grow beyond one chunk.
 *
 * Streams and errors.  Calls enqueue work on `stream` (a cudaStream_t, NULL
 * for the legacy default stream) and return without synchronising.
 * Argument and shape errors are returned synchronously and nothing is
 * enqueued.  Conditions found on the device never trap: a zero determinant
 * gives sign 0 and logabs = -inf; a non-finite local energy is written as
 * NaN; both are counted in a status word read by dq_last_device_status().
 * The library never calls exit() or abort().
 */
#ifndef DQMC_H
#define DQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DQ_OK = 0,
  DQ_ERR_ARG = 1,        /* null pointer, bad enum value, bad size      */
  DQ_ERR_SHAPE = 2,      /* unsupported molecule / ansatz dimensions     */
  DQ_ERR_CUDA = 3,       /* a CUDA runtime call failed                   */
  DQ_ERR_NONFINITE = 4,  /* reserved: reported via dq_last_device_status */
  DQ_ERR_WORKSPACE = 5,  /* workspace missing, too small or misaligned   */
  DQ_ERR_TIMEOUT = 6,    /* a bounded device wait gave up                */
  DQ_ERR_UNSUPPORTED = 7 /* not available in this precision or setting */
} dq_status;

typedef enum { DQ_FP64 = 0, DQ_FP32 = 1, DQ_BF16_MIXED = 2 } dq_precision;

/* Operation codes for dq_workspace_size. */
typedef enum {
  DQ_OP_EVAL = 0,
  DQ_OP_LOCAL_ENERGY = 1,
  DQ_OP_MCMC = 2,
  DQ_OP_GRAD = 3,
  DQ_OP_LOSS_WEIGHTS = 4,
  DQ_OP_MALA = 5,
  DQ_OP_AUTOTUNE = 6, /* dq_autotune_multi (batches only) */
  DQ_OP_NATGRAD = 7,  /* natural_gradient */
  DQ_OP_UPDATE = 8    /* param_update */
} dq_op;

/* Device status flags (dq_last_device_status). */
#define DQ_FLAG_SINGULAR 0x1u  /* some walker had psi = 0 (sign 0)          */
#define DQ_FLAG_NONFINITE 0x2u /* some local energy or gradient not finite   */
#define DQ_FLAG_TIMEOUT 0x4u   /* a bounded device wait gave up (kernel skipped its work) */

/* The molecule (Eq. 1).  Host memory; copied by dq_create. */
typedef struct {
  int32_t n_nuc;    /* M >= 1                        */
  const double* Z;  /* [M] nuclear charges           */
  const double* R;  /* [M][3] nuclear positions, bohr */
  int32_t n_up;     /* spin-up electrons, >= 1        */
  int32_t n_down;   /* spin-down electrons, >= 0      */
} dq_system;

/* Ansatz hyper-parameters (Sec. 3). */
typedef struct {
  int32_t width;      /* D: embedding width, multiple of 32, <= 512;
                       * a multiple of 64 in DQ_BF16_MIXED          */
  int32_t n_layers;   /* L >= 1 message-passing layers                */
  int32_t n_det;      /* K >= 1 determinant pairs                     */
  int32_t n_rbf;      /* Gaussian distance features, multiple of 8    */
  double rbf_cutoff;  /* rc: centre of the last Gaussian (bohr)       */
  int32_t use_jastrow;
  int32_t use_cusp;
  double cusp_alpha;  /* alpha of Eq. (25); 1 gives the Kato cusp     */
  int32_t full_det;   /* 0: psi = sum_p c_p det A^{up,p} det A^{down,p} (Eq. 21);
                       * 1: psi = sum_p c_p det A^p, one N x N matrix per p
                       *    whose row i comes from the orbital network and
                       *    envelopes of electron i's spin (Eq. 22); needs
                       *    N <= 32.  Other values: DQ_ERR_ARG.           */
  int32_t edge_update; /* 0: every layer filters the Gaussian features e(d);
                        * 1: edge embeddings iterated (Eq. 16, second case):
                        *    before layer l >= 1's filters,
                        *    f^l = f^{l-1} + tanh(U^{l,t} f^{l-1} + c^{l,t})
                        *    per edge type t, f^0 = e(d).  Other values:
                        *    DQ_ERR_ARG.                                   */
  int32_t el_init;     /* 0: f_i^0 = E_spin[spin of i] (Eq. 13, first case);
                        * 1: f_i^0 = W_e2 tanh(W_e1 x_i + b_e1) + b_e2 with
                        *    x_i = (r_i - R_1, ..., r_i - R_M) (Eq. 13,
                        *    second case); not rotation invariant.  Other
                        *    values: DQ_ERR_ARG.                            */
} dq_ansatz_cfg;

typedef struct dq_handle_s* dq_handle;

/* Create a handle on the current CUDA device.  Limits: n_up + n_down <= 64,
 * max(n_up, n_down) <= 32, n_nuc <= 64.  Allocates small device tables (the
 * only allocations of the library).  Returns DQ_ERR_SHAPE outside the limits. */
dq_status dq_create(const dq_system* sys, const dq_ansatz_cfg* cfg, int32_t precision, dq_handle* out);
dq_status dq_destroy(dq_handle h);

/* Number of parameters P of the flat vector described above. */
dq_status dq_param_count(dq_handle h, int64_t* P);

/* Largest walker chunk processed at once (default 4096), and a setter
 * (chunk >= 1).  Workspace sizes depend on min(B, chunk). */
dq_status dq_max_chunk(dq_handle h, int64_t* chunk);
dq_status dq_set_max_chunk(dq_handle h, int64_t chunk);

/* Workspace bytes needed by operation `op` (dq_op) for B walkers. */
dq_status dq_workspace_size(dq_handle h, int64_t B, int32_t op, size_t* bytes);

/* ansatz_eval: log|psi| and sign psi for B walkers (Sec. 3, Eqs. 7-8, 21,
 * 27-28).
 *   params  [P]        flat parameter vector
 *   r       [B][N][3]  electron positions, spin-sorted
 *   logabs  [B]  out   log|psi| (-inf where psi = 0)
 *   sign    [B]  out   +1, -1, or 0 where psi = 0                         */
dq_status ansatz_eval(dq_handle h, const void* params, const void* r, int64_t B, void* logabs, int8_t* sign,
                      void* ws, size_t ws_bytes, void* stream);

/* local_energy: E_loc = -1/2 sum_i (Lap_i log|psi| + |grad_i log|psi||^2) + V
 * (Sec. 4.2, Eq. 31), V = Coulomb potential of Eq. (1) plus the constant
 * nuclear repulsion sum_{I<J} Z_I Z_J / R_IJ.  Also writes logabs and sign.
 *   e_loc   [B]  out   NaN where psi = 0 or the result is not finite
 *   e_sum2  [2]  out   nullable, device double: sum_b E_loc, sum_b E_loc^2
 *                      (FP64 sums over the finite values)                  */
dq_status local_energy(dq_handle h, const void* params, const void* r, int64_t B, void* logabs, int8_t* sign,
                       void* e_loc, double* e_sum2, void* ws, size_t ws_bytes, void* stream);

/* mcmc_step: n_steps random-walk Metropolis steps (Sec. 5) on B walkers.
 * Step t = step_counter + s (s < n_steps) proposes r' = r + step_size * xi,
 * xi ~ N(0, 1)^(3N), and accepts iff log u < 2 (log|psi(r')| - log|psi(r)|)
 * (strict) and psi(r') != 0, u ~ U(0, 1).  xi and u are drawn from
 * Philox4x32-10 (Salmon et al., SC'11) with key = seed and counter
 * [walker, t mod 2^32, (tag << 24) | block, t >> 32], tag 1 for xi (Box-Muller
 * pairs of words (x0, x1), (x2, x3) of block q/4 give xi_q), tag 2 for u
 * (word x0 of block 0); uniforms are (x + 0.5) 2^-32.
 *   r        [B][N][3] in/out    positions
 *   logabs   [B]       in/out    log|psi| of r (as from ansatz_eval)
 *   n_accepted         nullable, device int64: set to the number of
 *                      accepted moves of this call                         */
dq_status mcmc_step(dq_handle h, const void* params, void* r, void* logabs, int64_t B, int32_t n_steps,
                    double step_size, uint64_t seed, uint64_t step_counter, int64_t* n_accepted, void* ws,
                    size_t ws_bytes, void* stream);

/* mcmc_step_dev: mcmc_step with the step counter in device memory:
 *   step_counter  device uint64, read by the call's kernels (step t =
 *                 *step_counter + s) and advanced by n_steps at its end.
 * Every other argument as for mcmc_step.  With the counter on the device a
 * captured CUDA graph of a VMC step (this call, local_energy, the loss
 * weights and grad_logpsi) replays successive Metropolis steps; the draws are
 * the same as mcmc_step's with step_counter = the counter's value. */
dq_status mcmc_step_dev(dq_handle h, const void* params, void* r, void* logabs, int64_t B, int32_t n_steps,
                        double step_size, uint64_t seed, uint64_t* step_counter, int64_t* n_accepted, void* ws,
                        size_t ws_bytes, void* stream);

/* mcmc_step_eloc: mcmc_step (the same Gaussian proposals of step_size, the
 * same uniforms and acceptance rule of step t = step_counter + s) whose
 * proposals are evaluated with value, 3N first derivatives and Laplacian
 * propagated together, as in local_energy, so that the local energy is carried
 * with every walker: after the call e_loc holds E_loc at the final positions,
 * and a VMC step needs one forward per walker instead of mcmc_step's value-only
 * forward followed by local_energy (no counterpart in the paper, which
 * evaluates the local energy after sampling; the sampled chain is the same).
 *   r        [B][N][3] in/out    positions
 *   logabs   [B]       in/out    log|psi| of r as local_energy gives it (the
 *                                acceptance compares it with the proposals'
 *                                log|psi| from the same forward)
 *   e_loc    [B]       in/out    E_loc at r, carried with r; valid only while
 *                                params do not change (after a parameter update,
 *                                recompute logabs and e_loc with local_energy)
 *   step_counter_dev   nullable, device uint64: read (step_counter ignored)
 *                      and advanced by n_steps, as in mcmc_step_dev
 *   n_accepted         nullable, device int64: accepted moves of this call
 * Workspace: dq_workspace_size(op = DQ_OP_MALA).  Asynchronous on `stream`. */
dq_status mcmc_step_eloc(dq_handle h, const void* params, void* r, void* logabs, void* e_loc, int64_t B,
                         int32_t n_steps, double step_size, uint64_t seed, uint64_t step_counter,
                         uint64_t* step_counter_dev, int64_t* n_accepted, void* ws, size_t ws_bytes, void* stream);

/* mala_step: n_steps Metropolis-adjusted Langevin steps (Sec. 5, the Langevin
 * sampler) on B walkers.  The paper names a correction that shortens electron
 * steps near the nuclei without giving it; here the drift of electron i,
 * v_i = d log|psi| / d r_i, is limited as (Umrigar, Nightingale, Runge,
 * J. Chem. Phys. 99, 2865 (1993), a = 1)
 *   vbar_i = v_i (sqrt(1 + 2 tau |v_i|^2) - 1) / (tau |v_i|^2).
 * Step t = step_counter + s proposes r' = r + tau vbar(r) + sqrt(tau) xi with
 * the normals xi of mcmc_step's step t, evaluates log|psi|, sign and
 * d log|psi| / d r at r' (value, 3N first derivatives and Laplacian
 * propagated together, as in local_energy), and accepts iff psi(r') != 0 and
 *   log u < 2 (log|psi(r')| - log|psi(r)|) + |xi|^2 / 2
 *           - |r - r' - tau vbar(r')|^2 / (2 tau)
 * with mcmc_step's uniform u of step t (FP64 arithmetic).
 *   r        [B][N][3] in/out    positions
 *   logabs   [B]       in/out    log|psi| of r
 *   grad     [B][N][3] in/out    d log|psi| / d r at r; grad_valid = 0 makes
 *                                the call compute it (and logabs) first, so
 *                                n_steps = 0 with grad_valid = 0 only sets up
 *                                logabs and grad at r
 *   e_loc    [B]       in/out    nullable: E_loc at r (as from local_energy),
 *                                carried with r (the proposal's evaluation
 *                                gives E_loc at r' at no extra cost; valid
 *                                while params do not change);
 *                                computed with grad when grad_valid = 0
 *   step_counter_dev   nullable, device uint64: if given, the step counter is
 *                      read from it (step_counter ignored) and advanced by
 *                      n_steps, as in mcmc_step_dev
 *   n_accepted         nullable, device int64: accepted moves of this call
 * tau > 0.  Workspace: dq_workspace_size(op = DQ_OP_MALA). */
dq_status mala_step(dq_handle h, const void* params, void* r, void* logabs, void* grad, void* e_loc,
                    int32_t grad_valid, int64_t B, int32_t n_steps, double tau, uint64_t seed, uint64_t step_counter,
                    uint64_t* step_counter_dev, int64_t* n_accepted, void* ws, size_t ws_bytes, void* stream);

/* grad_logpsi: parameter gradient of log|psi| (Sec. 4.1, Eq. 30).
 *   mode 0 (weighted): grad_out[P] = sum_b weights[b] d log|psi_b| / d theta
 *                      (weights [B] required);
 *   mode 1 (per walker): grad_out[B][P] = d log|psi_b| / d theta
 *                      (weights ignored, may be NULL).
 * Walkers with psi = 0 contribute zero.                                    */
dq_status grad_logpsi(dq_handle h, const void* params, const void* r, int64_t B, const void* weights,
                      int32_t mode, void* grad_out, void* ws, size_t ws_bytes, void* stream);

/* natural_gradient: the natural-gradient direction of the optimiser (Sec. 4,
 * "Optimizer"): the loss gradient g = G^T w (Eq. 30) preconditioned by the
 * damped Fisher information of |psi|^2 estimated from the walkers,
 *   delta = (Gc^T Gc / B + lambda I)^-1 g = Gc^T (Gc Gc^T / B + lambda I)^-1 w,
 * Gc = G minus its mean over the walkers (equal forms by the push-through
 * identity; the second, a B x B system, is the one solved).  The paper's
 * optimiser approximates this preconditioner by Kronecker factors; here it is
 * formed exactly in the walkers' space.
 *   G      [B][P] in   per-walker gradients d log|psi_b| / d theta, as from
 *                      grad_logpsi(mode = 1); not modified
 *   w      [B]    in   walker weights (vmc_loss_weights), so that G^T w is the
 *                      loss gradient
 *   lambda        damping (absorbs the factor 4 of the Fisher information): > 0
 *                 absolute; < 0 relative, |lambda| times the mean eigenvalue
 *                 tr(Gc Gc^T) / B^2 of Gc Gc^T / B (taken on the device)
 *   max_iter, tol conjugate-gradient iterations (at most max_iter; they stop on
 *                 the device once ||r|| <= tol ||w||)
 *   delta  [P]    out
 *   stats  [4]    nullable, device double out: iterations, final ||r|| / ||w||,
 *                 ||w||, the damping used
 * Gc Gc^T is formed on the tensor cores (3 x TF32 products); the system is
 * solved in FP64 with fixed-order reductions (deterministic).  FP32 and BF16
 * handles (DQ_ERR_UNSUPPORTED in FP64 mode); B >= 2.  Workspace:
 * dq_workspace_size(op = DQ_OP_NATGRAD, B), about 12 B P bytes. */
dq_status natural_gradient(dq_handle h, const void* G, const void* w, int64_t B, double lambda, int32_t max_iter,
                           double tol, void* delta, double* stats, void* ws, size_t ws_bytes, void* stream);

/* param_update: the parameter step of the optimiser around a direction such
 * as natural_gradient's, theta <- theta - lr s delta, with the step-length
 * limit s = min(1, max_norm / (lr ||delta||)) usual for natural-gradient steps
 * (max_norm <= 0: s = 1).  The paper's optimiser takes its step from a
 * third-party library; this is the plain form.
 *   params [P] in/out, delta [P] in (FP32 modes; DQ_ERR_UNSUPPORTED in FP64)
 *   stats  [2] device double out: ||delta||, s
 * ||delta|| is a fixed-order FP64 reduction.  Workspace:
 * dq_workspace_size(op = DQ_OP_UPDATE). */
dq_status param_update(dq_handle h, void* params, const void* delta, double lr, double max_norm, double* stats,
                       void* ws, size_t ws_bytes, void* stream);

/* Pseudopotentials (Eqs. 11 and 12): a nucleus with a
 * pseudopotential carries a local function V and non-local channels
 * W_0 .. W_lmax, each f(r) = sum_t beta_t r^(n_t - 2) exp(-alpha_t r^2).  The
 * handle's system then holds the valence electrons and effective charges; the
 * caller adds v_loc + v_nl to E_loc (and drops the Coulomb attraction of the
 * pseudopotential nuclei if its V replaces it). */
typedef struct {
  int32_t nucleus;     /* index of the nucleus */
  int32_t l_max;       /* non-local channels l = 0 .. l_max, l_max <= 3 */
  int32_t n_terms;     /* Gaussian terms of every radial function, 1 .. 4 */
  const double* coef;  /* host [(l_max + 2)][n_terms][3]: (beta, n, alpha), V first, then W_0 .. W_lmax */
} dq_pseudopotential;

/* pseudopotential_energy: per walker
 *   v_loc = sum_{i,I} V_I(r_iI),
 *   v_nl  = sum_{i,I,l} W_l(r_iI) (2l + 1) / 12 sum_k P_l(cos th_k) psi(r_i -> R_I + r_iI R_b u_k) / psi(r),
 * the angular integral of Eq. 12 summed over m by the addition
 * theorem and replaced by the 12-point icosahedral quadrature (vertices u_k
 * rotated by the walker's rotation R_b, cos th_k = (R_b u_k) . (r_i - R_I) / r_iI).
 * Every electron is displaced around every pseudopotential nucleus: B * N *
 * n_pp * 12 value-only evaluations of psi, in one batch.
 *   rot     [B][3][3] in   rotations (orthogonal; drawn by the caller, e.g. uniformly)
 *   logabs, sign [B] in    log|psi| and sign of r (as from ansatz_eval / local_energy)
 *   v_loc, v_nl  [B] out
 * 1 <= n_pp <= 8.  Workspace: dq_pp_workspace_size. */
dq_status dq_pp_workspace_size(dq_handle h, int64_t B, int32_t n_pp, size_t* bytes);
dq_status pseudopotential_energy(dq_handle h, const void* params, const void* r, int64_t B, int32_t n_pp,
                                 const dq_pseudopotential* pps, const void* rot, const void* logabs,
                                 const int8_t* sign, void* v_loc, void* v_nl, void* ws, size_t ws_bytes,
                                 void* stream);

/* vmc_loss_weights: clipped local energies and gradient weights (Sec. 4.4,
 * Eq. 30).  Centre mu = median of e_loc (mean of the two middle values for
 * even B), half-width = clip_k * mean |e_loc - mu|; E^_b = clamp(e_loc_b);
 * weights[b] = (2/B)(E^_b - mean_b E^_b), so that grad_logpsi(mode 0) with
 * these weights is the estimator of Eq. (30) on clipped energies.
 *   e_loc   [B]   in, finite values expected (B <= 65536)
 *   weights [B]   out
 *   stats   [4]   nullable, device double out: mu, half-width, mean E^,
 *                 mean of the unclipped e_loc                              */
dq_status vmc_loss_weights(dq_handle h, const void* e_loc, int64_t B, double clip_k, void* weights,
                           double* stats, void* ws, size_t ws_bytes, void* stream);

/* Clipping functions for vmc_loss_weights_clip (Sec. 4.4, "Gradient clipping"). */
enum { DQ_CLIP_HARD = 0, /* E^ = clamp(e, mu - sigma, mu + sigma) (von Glehn et al.)          */
       DQ_CLIP_LOG = 1   /* E^ = e inside |e - mu| <= sigma, else                              *
                          *      mu + sign(e - mu) sigma (1 + ln(|e - mu| / sigma)):           *
                          * the logarithmically growing soft window (Hermann et al.); value    *
                          * and slope are continuous at the window's edges                     */ };

/* vmc_loss_weights_clip: vmc_loss_weights with a choice of clipping function
 * (sigma = the half-width clip_k * MAD, mu = the median).  clip_mode outside
 * DQ_CLIP_HARD / DQ_CLIP_LOG returns DQ_ERR_ARG.  Other arguments, workspace
 * and stats as for vmc_loss_weights; DQ_CLIP_HARD gives the same results.   */
dq_status vmc_loss_weights_clip(dq_handle h, const void* e_loc, int64_t B, double clip_k, int32_t clip_mode,
                                void* weights, double* stats, void* ws, size_t ws_bytes, void* stream);

/* vmc_loss_weights_noalloc: the same weights and stats as vmc_loss_weights,
 * for callers that cannot allocate device memory and so cannot supply a
 * workspace (for example a plugin whose host framework owns all device
 * allocations, or a service that must not allocate after start-up).  The
 * paper has no counterpart; this is a deployment convenience.
 * The sort scratch is a fixed 512 KB array inside the library (one per GPU
 * that loads it, kept until exit), so B must not exceed 65536; larger B
 * returns DQ_ERR_SHAPE and nothing is enqueued.  No call allocates.
 * The first call on a device (with that device current) looks up the
 * array's device address and caches it for the life of the process; it may
 * load the library's module, so make it before any stream capture.  A device
 * reset (cudaDeviceReset, or a reset of the primary context) destroys the
 * array and invalidates the cached address, as it does the handles' device
 * buffers: do not call this entry point on that device after a reset.  With
 * the handle's profiling on (dq_profile_enable) the launch is timed as the
 * loss_weights kind.  All calls on a device share the array: calls
 * whose kernels overlap on the GPU (unordered streams) race and give wrong
 * results.  Arguments as for vmc_loss_weights.                              */
dq_status vmc_loss_weights_noalloc(dq_handle h, const void* e_loc, int64_t B, double clip_k, void* weights,
                                   double* stats, void* stream);

/* Reads and clears the device status flags (DQ_FLAG_*) accumulated since the
 * last read.  Synchronises `stream`. */
dq_status dq_last_device_status(dq_handle h, void* stream, uint32_t* flags);

/* Number of determinant matrices factorised in FP64 since the last read
 * (then cleared; synchronises `stream`).  In the FP32 modes every matrix is
 * first factorised in FP32 and near-nodal ones are redone in FP64, which this
 * counts: value-only calls (ansatz_eval, mcmc_step) when the condition
 * estimate of the row-equilibrated matrix exceeds 10000 (below that the FP32
 * log|det| is corrected by the trace of the factorisation residual against
 * the FP32 inverse); local_energy, for determinant blocks of at most 28
 * electrons, when it exceeds 1e5 or when the iterative refinement of the FP32
 * inverse (double-float, at most four steps) does not bring the largest
 * residual entry below 1e-4 (otherwise the tangent products run in
 * double-float on the FP32 pipes).
 * local_energy with larger blocks takes FP64 for every matrix (not counted).
 * Always 0 in FP64 mode, where every matrix is FP64. */
dq_status dq_fp64_matrix_count(dq_handle h, void* stream, int64_t* count);

/* Test support: the BF16 tensor-core GEMM used by the embedding layers in
 * DQ_BF16_MIXED mode, exposed so that it can be checked on its own.
 * Y[r][n] = sum_k X[r][k] W[n][k] + (r % bias_period == 0 ? bias[n] : 0);
 * X [rows][K] (row stride ldx) and W [n_out][K] BF16 device arrays, 16-byte
 * aligned, K a multiple of 64, ldx a multiple of 8; bias FP32 [n_out] or
 * NULL; Y FP32 [rows][ldy].  status: device uint32 receiving DQ_FLAG_TIMEOUT
 * if a bounded wait inside the kernel gave up.  Enqueued on `stream`. */
dq_status dq_test_gemm_bf16(const void* X, int64_t rows, int32_t K, int64_t ldx, const void* W, int32_t n_out,
                            const float* bias, int32_t bias_period, float* Y, int64_t ldy, uint32_t* status,
                            void* stream);

/* Test support (not part of the method): the FP32-accurate tensor-core GEMM
 * of the FP32 mode on its own.  Y[r][n] = sum_k X[r][k] W[n][k] (+ bias[n]
 * when r % bias_period == 0), computed as three TF32 tensor-core products of
 * the operands split into TF32 high and low parts (x_hi w_hi + x_hi w_lo +
 * x_lo w_hi; relative error about 2^-21 of sum_k |x_k w_k|).  X FP32 device
 * [rows][ldx], K a multiple of 4, ldx a multiple of 4, X and W 16-byte
 * aligned; W FP32 device [n_out][K]; wsplit: device FP32 scratch of
 * 2 * n_out * K elements that receives the split W; Y FP32 [rows][ldy];
 * status as for dq_test_gemm_bf16.  Enqueued on `stream`. */
dq_status dq_test_gemm_tf32x3(const float* X, int64_t rows, int32_t K, int64_t ldx, const float* W, int32_t n_out,
                              const float* bias, int32_t bias_period, float* Y, int64_t ldy, float* wsplit,
                              uint32_t* status, void* stream);

/* ---- Batches of molecules ------------------------------------------------
 * A batch holds up to DQ_MAX_BATCH molecules, each with its own system,
 * ansatz sizes and parameter vector, in one precision (DQ_FP32 or
 * DQ_BF16_MIXED) and with equal numbers of layers.  The walkers of all
 * molecules, uneven electron counts included, go through every step of the
 * forward pass (Sec. 3 and Sec. 4.2), the Metropolis sampler (Sec. 5) and the
 * loss weights (Sec. 4.4) in one kernel launch per step: each launch carries
 * a table with every molecule's dimensions, parameters and buffers, and the
 * tensor-core GEMMs of a step run as one persistent launch whose tiles cover
 * all molecules.  Walkers are processed in `rounds` chunks (molecule m takes
 * ceil(B[m] / rounds) walkers per chunk); 0, the default, picks the fewest
 * chunks of at most dq_max_chunk walkers of each molecule.  Each molecule's
 * results equal those of the single-molecule calls on its own handle with the
 * same inputs (the single-molecule calls launch the same kernels with a
 * one-entry table): log|psi|, sign and E_loc bit for bit, and the Metropolis
 * draws of molecule m are those of mcmc_step with the same seed and step
 * counter.  grad_logpsi_multi runs the reverse pass molecule by molecule.
 * Array arguments (params, r, B, logabs, ...) are HOST arrays of n_mol
 * entries; entry m is a device pointer (or count) for molecule m, laid out as
 * in the single-molecule call.  Workspace: dq_multi_workspace_size with the
 * same B and op (DQ_OP_EVAL, _LOCAL_ENERGY, _MCMC, _GRAD, _LOSS_WEIGHTS). */
#define DQ_MAX_BATCH 8
typedef struct dq_multi_s* dq_multi;
dq_status dq_create_multi(int32_t n_mol, const dq_system* systems, const dq_ansatz_cfg* cfgs, int32_t precision,
                          dq_multi* out);
dq_status dq_destroy_multi(dq_multi m);
/* Borrowed handle of molecule k (parameter count and layout, single-molecule
 * calls); owned by the batch, valid until dq_destroy_multi. */
dq_status dq_multi_handle(dq_multi m, int32_t k, dq_handle* h);
dq_status dq_multi_set_rounds(dq_multi m, int32_t rounds);
dq_status dq_multi_rounds(dq_multi m, int32_t* rounds);
dq_status dq_multi_workspace_size(dq_multi m, const int64_t* B, int32_t op, size_t* bytes);
dq_status ansatz_eval_multi(dq_multi m, const void* const* params, const void* const* r, const int64_t* B,
                            void* const* logabs, int8_t* const* sign, void* ws, size_t ws_bytes, void* stream);
/* e_sum2: nullable host array; entry m nullable, device double[2] of molecule m. */
dq_status local_energy_multi(dq_multi m, const void* const* params, const void* const* r, const int64_t* B,
                             void* const* logabs, int8_t* const* sign, void* const* e_loc, double* const* e_sum2,
                             void* ws, size_t ws_bytes, void* stream);
/* One step counter for the batch: host step_counter, or the device counter
 * step_counter_dev (nullable) as in mcmc_step_dev.  n_accepted: nullable host
 * array of nullable device int64 counters, one per molecule. */
dq_status mcmc_step_multi(dq_multi m, const void* const* params, void* const* r, void* const* logabs,
                          const int64_t* B, int32_t n_steps, double step_size, uint64_t seed, uint64_t step_counter,
                          uint64_t* step_counter_dev, int64_t* const* n_accepted, void* ws, size_t ws_bytes,
                          void* stream);
/* Weighted gradient (grad_logpsi mode 0) of every molecule. */
dq_status grad_logpsi_multi(dq_multi m, const void* const* params, const void* const* r, const int64_t* B,
                            const void* const* weights, void* const* grad_out, void* ws, size_t ws_bytes,
                            void* stream);
/* stats: nullable host array; entry m nullable, device double[4] as in vmc_loss_weights. */
dq_status vmc_loss_weights_multi(dq_multi m, const void* const* e_loc, const int64_t* B, double clip_k,
                                 void* const* weights, double* const* stats, void* ws, size_t ws_bytes,
                                 void* stream);

/* Tile shape of one handle (no counterpart in the paper): msg_ib = receivers
 * per warp task of the jet message kernel (its register tile is msg_ib x 4
 * channels; 8 or 4, 0 restores the default 8).  Results do not depend on it. */
dq_status dq_set_msg_tile(dq_handle h, int32_t msg_ib);
dq_status dq_msg_tile(dq_handle h, int32_t* msg_ib);

/* Jet message kernel of the separate layer path (Eq. 17 with the product rule;
 * no counterpart in the paper): mode 1 the general kernel (a warp task holds
 * msg_ib receivers x 4 channels, the senders' node channels streamed through
 * shared memory, the filter tables of all pairs resident); mode 2 the
 * sender-tiled kernel (one spin block of senders at a time: a warp task holds
 * their node channels for up to 11 channels in registers and runs over every
 * receiver; FP32 and BF16 modes, width a multiple of 32, at most 48
 * electrons, 24 per spin); mode 0 (the default) is mode 2 above 16 electrons
 * where supported and mode 1 elsewhere.  Layers whose node channels are the
 * spin-embedding constants always take the general kernel.  Mode 2 on a DQ_FP64
 * handle: DQ_ERR_UNSUPPORTED; other modes: DQ_ERR_ARG.  Both kernels compute
 * the same messages within FP32 rounding (different summation orders).
 * dq_msg_kernel reports the kernel the handle's jet layers take on the
 * separate path (1 or 2). */
dq_status dq_set_msg_kernel(dq_handle h, int32_t mode);
dq_status dq_msg_kernel(dq_handle h, int32_t* mode);

/* Kernels of the jet layers (Eqs. 17-18) of local_energy and mala_step (no
 * counterpart in the paper): mode 1 runs each layer's messages, update map W_g
 * and residual tanh update as one kernel whose messages are the tensor-core
 * A operand and never reach memory; mode 2 runs them as the message kernel,
 * the W_g GEMM and the update kernel, with the messages in the workspace;
 * mode 0 (the default) is mode 1 where the handle supports it and mode 2
 * elsewhere.  Mode 1 needs DQ_FP32 or DQ_BF16_MIXED (whose fused kernel takes
 * the electron-electron messages and W_g as BF16 operands), width 128, at
 * most 16 electrons (8 per spin) and 8 nuclei: DQ_ERR_UNSUPPORTED otherwise.  Both modes compute the
 * same quantities within the FP32 mode's rounding (the sums run in different
 * orders).  The workspace size depends on the mode (mode 2 adds the message
 * buffer): query dq_workspace_size after setting it.  dq_layer_kernel reports
 * 1 if the jet layers currently run fused, else 0. */
dq_status dq_set_layer_kernel(dq_handle h, int32_t mode);
dq_status dq_layer_kernel(dq_handle h, int32_t* fused);

/* Warps per CTA of the grouped determinant kernels (no counterpart in the
 * paper; the matrices of Eqs. 21-22, one per warp): 4 (the default) or 2,
 * DQ_ERR_ARG otherwise.  Results do not depend on it.  dq_tile_set reports the
 * handle's current tile set: walker chunk, msg_ib, layer kernels (1 fused,
 * 2 separate) and determinant warps per CTA (host outputs, non-null). */
dq_status dq_set_det_warps(dq_handle h, int32_t warps);
dq_status dq_tile_set(dq_handle h, int64_t* max_chunk, int32_t* msg_ib, int32_t* layer_kernel, int32_t* det_warps);

/* dq_autotune times local_energy on the given walkers for every candidate of
 *   layer kernels  fused, separate   (dq_set_layer_kernel 1 or 2; the fused
 *                                      one only where supported, the separate
 *                                      one only if ws_bytes holds its message
 *                                      buffer),
 *   walker chunk   4096, 2048        (dq_set_max_chunk: the M extent of every
 *                                      GEMM, the grid of every other kernel),
 *   msg_ib         8, 4              (separate message kernel only),
 *   det warps      4, 2              (dq_set_det_warps; with the 4096 chunk),
 * one warm-up and two timed calls each (CUDA events on `stream`, host waits),
 * and keeps the fastest; workspace: at least dq_workspace_size(op =
 * DQ_OP_LOCAL_ENERGY) for a chunk of min(B, 4096) walkers plus 9 B per
 * walker.  The chosen set is cached in the process per molecule size
 * (electrons, spin-up electrons, nuclei), ansatz shape (width, layers,
 * determinants, radial features, variant flags), precision and B: a later
 * call with the same key applies the cached set without timing (best_ms then
 * reports the cached time).  Synchronises; not for use inside a stream
 * capture.  best_ms: nullable host double. */
dq_status dq_autotune(dq_handle h, const void* params, const void* r, int64_t B, void* ws, size_t ws_bytes,
                      void* stream, double* best_ms);

/* Autotuner of a batch's tile shapes (no counterpart in the paper; the
 * batching it serves is the paper's many-molecule use of one program): times
 * local_energy_multi on the given walkers for every candidate of
 *   rounds   1, 2, 3, 4   (walkers per launch: the M extent of every GEMM and
 *                          the grid of every other kernel), and
 *   msg_ib   8, 4         (receivers per warp task of the jet message kernel:
 *                          its register tile of msg_ib x 4 channels),
 * one warm-up and two timed calls each (CUDA events on `stream`, host waits),
 * then, at the winning pair, the determinant kernels' warps per CTA (4, 2),
 * and keeps the fastest in the batch (later calls use it; dq_multi_tuning
 * and dq_multi_tile_set report it).  Candidates whose workspace exceeds
 * ws_bytes are skipped.
 * Workspace: dq_multi_workspace_size(op = DQ_OP_AUTOTUNE) covers all
 * candidates and the timing outputs.  Synchronises; not for use inside a
 * stream capture.  best_ms: nullable host double, the winner's time. */
dq_status dq_autotune_multi(dq_multi m, const void* const* params, const void* const* r, const int64_t* B, void* ws,
                            size_t ws_bytes, void* stream, double* best_ms);
dq_status dq_multi_tuning(dq_multi m, int32_t* rounds, int32_t* msg_ib);
/* The batch's tile set: rounds, msg_ib, the number of molecules whose jet
 * layers run fused (dq_set_layer_kernel mode 1) and the determinant warps per
 * CTA (host outputs, non-null). */
dq_status dq_multi_tile_set(dq_multi m, int32_t* rounds, int32_t* msg_ib, int32_t* fused_layers,
                            int32_t* det_warps);

/* Measurement support (not part of the method): enqueues on `stream` one
 * launch of a kernel that only issues fused multiply-adds on the CUDA cores,
 * kind 0 FP32 (FFMA), kind 1 FP64 (DFMA): `blocks` blocks of 256 threads,
 * each thread `iters` x 128 FMAs in 8 independent chains.  The caller times
 * the launch (CUDA events on `stream`) and divides *flops (host double, the
 * launch's floating-point operations, 2 per FMA) by the time: the measured
 * peak FMA rate against which kernels bound by CUDA-core arithmetic are
 * reported.  sink: device buffer of at least `blocks` elements of the kind's
 * type (never written for the probe's inputs).  DQ_ERR_ARG on bad sizes or
 * kind. */
dq_status dq_fma_rate_probe(int32_t kind, int32_t blocks, int32_t iters, void* sink, void* stream, double* flops);

/* Human-readable name of a status code (static string). */
const char* dq_status_string(dq_status s);

/* Measurement support (not part of the method): when enabled, every kernel
 * launch of the handle is bracketed by two CUDA events recorded on the
 * launching stream (from a pool of 32768 events created at the first
 * enable, host-side driver objects only).  dq_profile_read synchronises on
 * the recorded events and returns, for one kernel kind (0 <= kind <
 * dq_profile_kind_count()), the summed device time in ms and the launch
 * count since the last reset; it returns DQ_ERR_WORKSPACE if the pool ran
 * out (later launches were not timed).  Kind names: dq_profile_kind_name. */
dq_status dq_profile_enable(dq_handle h, int32_t on);
dq_status dq_profile_reset(dq_handle h);
dq_status dq_profile_read(dq_handle h, int32_t kind, double* total_ms, int64_t* launches);
const char* dq_profile_kind_name(int32_t kind);
int32_t dq_profile_kind_count(void);

#ifdef __cplusplus
}
#endif

#endif /* DQMC_H */
