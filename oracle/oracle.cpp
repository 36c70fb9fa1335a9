// FP64 CPU oracle of the DeepQMC-style VMC hot path.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
// CUDA library is checked against.  Only the test-suite, the smoke check and
// the CPU-baseline leg of the benchmark load it; the library never does.  It
// shares no code, header or table with the CUDA path.
//
// What it computes (DeepQMC paper, Sec. 2-5):
//   * log|psi| and sign psi of the ansatz instance below, for one walker at a
//     time, straight from the definitions:
//       - graph convolution messages, Eq. (17), normalised by the number of
//         edges, and the concatenating residual update, Eq. (18) (Sec. 3.1);
//       - spin-only initial electron embedding, Eq. (13) first case, or
//         (el_init) an MLP of the electron-nucleus difference vectors,
//         Eq. (13) second case: f^0_i = W_e2 tanh(W_e1 x_i + b_e1) + b_e2,
//         x_i = (r_i - R_1, ..., r_i - R_M);
//       - edge features: Gaussian expansion of the distance, reused in every
//         layer, Eqs. (15)-(16) first case, or (edge_update) updated from
//         layer to layer, Eq. (16) second case, with the residual map
//         f^l = f^{l-1} + tanh(U^{l,t} f^{l-1} + c^{l,t}) per edge type;
//       - many-body orbitals kappa(f_i^L) (linear), Eq. (19), times isotropic
//         Slater envelopes (alpha = 1, one exponential per nucleus), Eq. (20);
//       - spin-factorised determinant pairs, Eq. (21), or (full_det) one
//         determinant of all N electrons per p, Eq. (22), whose rows come
//         from the orbital network of the electron's spin;
//       - learnable Jastrow factor, Eq. (24), and electron cusp, Eq. (25);
//       - log-domain evaluation with log-sum-exp over determinants,
//         Eqs. (27)-(28) (Sec. 3.5);
//   * the local energy, Eq. (31), with the potential of Eq. (1) plus the
//     constant nuclear repulsion.  The 3N second derivatives are taken one
//     coordinate at a time with hyper-dual numbers (Fike & Alonso, 2011),
//     seeding eps1 = eps2 = e_x: this is the "serial" forward-mode Laplacian
//     of Appendix A.2, not the GPU's batched propagation;
//   * directional derivatives of log|psi| in parameter space with dual
//     numbers (for the gradient estimator, Eq. (30));
//   * one random-walk Metropolis step (Sec. 5) on random draws passed in.
//
// Determinants: LU factorisation with partial pivoting on |value|.
//
// The base scalar is FP64.  Compiling with -DORACLE_REAL=float gives the same
// algorithm in FP32; that build exists only to measure the rounding floor of
// an FP32 evaluation of the method (it is never a reference).
// Parity status: every function here is pinned by tests (closed forms,
// invariants, finite differences, brute force); see the test-suite.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_REAL
#define ORACLE_REAL double
#endif
typedef ORACLE_REAL real;

namespace {

// ---------------------------------------------------------------------------
// Number types
// ---------------------------------------------------------------------------
// Hyper-dual number x = v + a e1 + b e2 + ab e1e2, e1^2 = e2^2 = 0.
struct HD {
  real v = 0, a = 0, b = 0, ab = 0;
  HD() = default;
  HD(real x) : v(x) {}
  HD(real v_, real a_, real b_, real ab_) : v(v_), a(a_), b(b_), ab(ab_) {}
};
inline HD operator+(const HD& x, const HD& y) { return {x.v + y.v, x.a + y.a, x.b + y.b, x.ab + y.ab}; }
inline HD operator-(const HD& x, const HD& y) { return {x.v - y.v, x.a - y.a, x.b - y.b, x.ab - y.ab}; }
inline HD operator-(const HD& x) { return {-x.v, -x.a, -x.b, -x.ab}; }
inline HD operator*(const HD& x, const HD& y) {
  return {x.v * y.v, x.v * y.a + x.a * y.v, x.v * y.b + x.b * y.v,
          x.v * y.ab + x.a * y.b + x.b * y.a + x.ab * y.v};
}
inline HD& operator+=(HD& x, const HD& y) { x = x + y; return x; }
inline HD& operator-=(HD& x, const HD& y) { x = x - y; return x; }
// f(x) for a scalar function with value f, first derivative d1, second d2.
inline HD chain(const HD& x, real f, real d1, real d2) {
  return {f, d1 * x.a, d1 * x.b, d1 * x.ab + d2 * x.a * x.b};
}
inline HD inv(const HD& x) { real i = 1.0 / x.v; return chain(x, i, -i * i, 2 * i * i * i); }
inline HD operator/(const HD& x, const HD& y) { return x * inv(y); }
inline HD exp(const HD& x) { real e = std::exp(x.v); return chain(x, e, e, e); }
inline HD log(const HD& x) { return chain(x, std::log(x.v), 1.0 / x.v, -1.0 / (x.v * x.v)); }
inline HD sqrt(const HD& x) { real s = std::sqrt(x.v); return chain(x, s, 0.5 / s, -0.25 / (s * x.v)); }
inline HD tanh(const HD& x) { real t = std::tanh(x.v); real d = 1 - t * t; return chain(x, t, d, -2 * t * d); }
inline real val(const HD& x) { return x.v; }

// Dual number x = v + d e, e^2 = 0.
struct Dual {
  real v = 0, d = 0;
  Dual() = default;
  Dual(real x) : v(x) {}
  Dual(real v_, real d_) : v(v_), d(d_) {}
};
inline Dual operator+(const Dual& x, const Dual& y) { return {x.v + y.v, x.d + y.d}; }
inline Dual operator-(const Dual& x, const Dual& y) { return {x.v - y.v, x.d - y.d}; }
inline Dual operator-(const Dual& x) { return {-x.v, -x.d}; }
inline Dual operator*(const Dual& x, const Dual& y) { return {x.v * y.v, x.v * y.d + x.d * y.v}; }
inline Dual& operator+=(Dual& x, const Dual& y) { x = x + y; return x; }
inline Dual& operator-=(Dual& x, const Dual& y) { x = x - y; return x; }
inline Dual chain(const Dual& x, real f, real d1) { return {f, d1 * x.d}; }
inline Dual inv(const Dual& x) { real i = 1.0 / x.v; return chain(x, i, -i * i); }
inline Dual operator/(const Dual& x, const Dual& y) { return x * inv(y); }
inline Dual exp(const Dual& x) { real e = std::exp(x.v); return chain(x, e, e); }
inline Dual log(const Dual& x) { return chain(x, std::log(x.v), 1.0 / x.v); }
inline Dual sqrt(const Dual& x) { real s = std::sqrt(x.v); return chain(x, s, 0.5 / s); }
inline Dual tanh(const Dual& x) { real t = std::tanh(x.v); return chain(x, t, 1 - t * t); }
inline real val(const Dual& x) { return x.v; }

inline real val(real x) { return x; }
using std::exp;
using std::log;
using std::sqrt;
using std::tanh;

template <class T> inline T absv(const T& x) { return val(x) < 0 ? -x : x; }

// ---------------------------------------------------------------------------
// System, hyper-parameters and the flat parameter layout
// ---------------------------------------------------------------------------
}  // namespace

extern "C" {
// Mirrors the Python-side ctypes structure in oracle/__init__.py.
struct OracleSpec {
  int32_t n_nuc;
  const real* Z;  // [n_nuc]
  const real* R;  // [n_nuc][3], bohr
  int32_t n_up, n_dn;
  int32_t D, L, K, Q;  // width, layers, determinant pairs, Gaussian features
  real rc;           // Gaussian feature cutoff
  int32_t use_jastrow, use_cusp;
  real alpha;        // cusp width
  int32_t full_det;  // 0: det A^up det A^down per p (Eq. 21); 1: det of the N x N A^p (Eq. 22)
  int32_t edge_update;  // 1: edge embeddings iterated between layers (Eq. 16, second case)
  int32_t el_init;      // 1: initial embeddings from electron-nucleus differences (Eq. 13, second case)
};
}

namespace {

// Offsets of every block of the flat parameter vector.  Order: E_spin[2][D]
// (or, with el_init, W_e1[D][3M], b_e1[D], W_e2[D][D], b_e2[D]);
// per layer: W_h[D][D], ([U[Q][Q], c[Q] when edge embeddings are iterated and
// l >= 1], W1[D][Q], b1[D], W2[D][D], b2[D]) for the
// same-spin, opposite-spin and electron-nucleus edge types, Y[M][D],
// W_g[D][3D], b_g[D]; per spin (up, down): W_o[K n_c][D], b_o[K n_c],
// omega[K n_c][M], zeta[K n_c][M]; c[K]; W_J1[D][D], b_J1[D], w_J2[D].
// n_c, the orbitals per determinant, is n_s (the electrons of that spin)
// for spin-factorised determinants and N for the full determinant; row
// p n_c + k of a spin's block is orbital k of determinant p.
struct Layout {
  int64_t E_spin = -1, W_e1 = -1, b_e1 = -1, W_e2 = -1, b_e2 = -1;
  struct Layer {
    int64_t W_h, U[3], c[3], W1[3], b1[3], W2[3], b2[3], Y, W_g, b_g;
  };
  std::vector<Layer> layer;
  int64_t W_o[2], b_o[2], omega[2], zeta[2], c, W_J1, b_J1, w_J2, total;

  explicit Layout(const OracleSpec& s) {
    const int64_t D = s.D, Q = s.Q, M = s.n_nuc, K = s.K;
    int64_t o = 0;
    if (s.el_init) {
      W_e1 = o; o += D * 3 * M;
      b_e1 = o; o += D;
      W_e2 = o; o += D * D;
      b_e2 = o; o += D;
    } else {
      E_spin = o; o += 2 * D;
    }
    layer.resize(s.L);
    for (int l = 0; l < s.L; ++l) {
      Layer& y = layer[l];
      y.W_h = o; o += D * D;
      for (int t = 0; t < 3; ++t) {
        y.U[t] = y.c[t] = -1;
        if (s.edge_update && l > 0) {
          y.U[t] = o; o += Q * Q;
          y.c[t] = o; o += Q;
        }
        y.W1[t] = o; o += D * Q;
        y.b1[t] = o; o += D;
        y.W2[t] = o; o += D * D;
        y.b2[t] = o; o += D;
      }
      y.Y = o; o += M * D;
      y.W_g = o; o += D * 3 * D;
      y.b_g = o; o += D;
    }
    const int64_t N = s.n_up + s.n_dn;
    const int64_t nc[2] = {s.full_det ? N : s.n_up, s.full_det ? N : s.n_dn};
    for (int sg = 0; sg < 2; ++sg) {
      W_o[sg] = o; o += K * nc[sg] * D;
      b_o[sg] = o; o += K * nc[sg];
      omega[sg] = o; o += K * nc[sg] * M;
      zeta[sg] = o; o += K * nc[sg] * M;
    }
    c = o; o += K;
    W_J1 = o; o += D * D;
    b_J1 = o; o += D;
    w_J2 = o; o += D;
    total = o;
  }
};

// ---------------------------------------------------------------------------
// Pieces of the ansatz
// ---------------------------------------------------------------------------
// y = W x (+ b), W row-major [n_out][n_in].
template <class T>
void affine(const T* W, const T* b, const T* x, int n_out, int n_in, T* y) {
  for (int a = 0; a < n_out; ++a) {
    T acc = b ? b[a] : T(0.0);
    const T* w = W + (int64_t)a * n_in;
    for (int c = 0; c < n_in; ++c) acc += w[c] * x[c];
    y[a] = acc;
  }
}

// Gaussian expansion of a distance: e_q = exp(-(d - mu_q)^2 / (2 s^2)),
// mu_q = q rc / (Q-1), s = rc / (Q-1) (Sec. 3.1, edge features).
template <class T>
void gaussian_features(const T& d, int Q, real rc, T* e) {
  const real s = rc / (Q - 1);
  for (int q = 0; q < Q; ++q) {
    T x = d - T(q * s);
    e[q] = exp(x * x * T(-0.5 / (s * s)));
  }
}

// Edge filter w(e) = W2 tanh(W1 e + b1) + b2.
template <class T>
void edge_filter(const T* th, const Layout::Layer& y, int t, const T* e, int D, int Q, T* out) {
  std::vector<T> h(D);
  affine(th + y.W1[t], th + y.b1[t], e, D, Q, h.data());
  for (int a = 0; a < D; ++a) h[a] = tanh(h[a]);
  affine(th + y.W2[t], th + y.b2[t], h.data(), D, D, out);
}

// sign and log|det| of an n x n matrix by LU with partial pivoting.
// A 0 x 0 determinant is 1.  A zero pivot gives sign 0, log|det| = -inf.
template <class T>
void slogdet(std::vector<T> A, int n, int* sign, T* logabs) {
  int sg = 1;
  T la(0.0);
  for (int j = 0; j < n; ++j) {
    int p = j;
    for (int i = j + 1; i < n; ++i)
      if (std::abs(val(A[i * n + j])) > std::abs(val(A[p * n + j]))) p = i;
    if (val(A[p * n + j]) == 0.0) {
      *sign = 0;
      *logabs = T(-std::numeric_limits<real>::infinity());
      return;
    }
    if (p != j) {
      for (int k = 0; k < n; ++k) std::swap(A[p * n + k], A[j * n + k]);
      sg = -sg;
    }
    const T piv = A[j * n + j];
    for (int i = j + 1; i < n; ++i) {
      const T f = A[i * n + j] / piv;
      for (int k = j + 1; k < n; ++k) A[i * n + k] -= f * A[j * n + k];
    }
    if (val(piv) < 0) sg = -sg;
    la += log(absv(piv));
  }
  *sign = sg;
  *logabs = la;
}

template <class T>
struct Walker {
  int sign = 0;
  T logabs;
};

// log|psi| and sign psi of one walker.  r: [N][3].  Optional debug outputs:
// Edge embedding of layer l of an edge of type t at distance d (Eq. 16): the
// Gaussian features, then, when iterated, l residual updates
// f <- f + tanh(U^{l',t} f + c^{l',t}) for l' = 1 .. l.
template <class T>
void edge_embedding(const OracleSpec& s, const Layout& lay, const T* th, int l, int t, const T& d, T* e) {
  gaussian_features(d, s.Q, s.rc, e);
  if (!s.edge_update) return;
  std::vector<T> a(s.Q);
  for (int lp = 1; lp <= l; ++lp) {
    affine(th + lay.layer[lp].U[t], th + lay.layer[lp].c[t], e, s.Q, s.Q, a.data());
    for (int q = 0; q < s.Q; ++q) e[q] = e[q] + tanh(a[q]);
  }
}

// f_out [N][D] final embeddings, A_out [2][K][nmax][nmax] orbital matrices.
template <class T>
Walker<T> log_psi(const OracleSpec& s, const Layout& lay, const T* th, const T* r,
                  real* f_out = nullptr, real* A_out = nullptr) {
  const int N = s.n_up + s.n_dn, M = s.n_nuc, D = s.D, Q = s.Q, K = s.K;
  auto spin = [&](int i) { return i < s.n_up ? 0 : 1; };

  // Distances (Sec. 3.1, graph representation).
  std::vector<T> dee(N * N, T(0.0)), den(N * M);
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j) {
      T acc(0.0);
      for (int x = 0; x < 3; ++x) {
        T dx = r[3 * i + x] - r[3 * j + x];
        acc += dx * dx;
      }
      dee[i * N + j] = dee[j * N + i] = sqrt(acc);
    }
  for (int i = 0; i < N; ++i)
    for (int I = 0; I < M; ++I) {
      T acc(0.0);
      for (int x = 0; x < 3; ++x) {
        T dx = r[3 * i + x] - T(s.R[3 * I + x]);
        acc += dx * dx;
      }
      den[i * M + I] = sqrt(acc);
    }

  // Initial embeddings: f_i^0 = E_spin[sigma_i] (Eq. 13, first case), or an MLP
  // of the difference vectors r_i - R_I (Eq. 13, second case).
  std::vector<T> f(N * D);
  if (s.el_init) {
    std::vector<T> x(3 * M), hid(D);
    for (int i = 0; i < N; ++i) {
      for (int I = 0; I < M; ++I)
        for (int c = 0; c < 3; ++c) x[3 * I + c] = r[3 * i + c] - T(s.R[3 * I + c]);
      affine(th + lay.W_e1, th + lay.b_e1, x.data(), D, 3 * M, hid.data());
      for (int a = 0; a < D; ++a) hid[a] = tanh(hid[a]);
      affine(th + lay.W_e2, th + lay.b_e2, hid.data(), D, D, &f[i * D]);
    }
  } else {
    for (int i = 0; i < N; ++i)
      for (int a = 0; a < D; ++a) f[i * D + a] = th[lay.E_spin + spin(i) * D + a];
  }

  std::vector<T> e(Q), w(D), z(N * D), m(3 * D), u(D);
  const int n_same[2] = {s.n_up, s.n_dn}, n_opp[2] = {s.n_dn, s.n_up};
  for (int l = 0; l < s.L; ++l) {
    const Layout::Layer& y = lay.layer[l];
    for (int j = 0; j < N; ++j) affine(th + y.W_h, (const T*)nullptr, &f[j * D], D, D, &z[j * D]);
    // Edge filters of the same-spin / opposite-spin e-e edges, per unordered pair.
    std::vector<T> wee(N * N * D, T(0.0));
    for (int i = 0; i < N; ++i)
      for (int j = i + 1; j < N; ++j) {
        const int t = spin(i) == spin(j) ? 0 : 1;
        edge_embedding(s, lay, th, l, t, dee[i * N + j], e.data());
        edge_filter(th, y, t, e.data(), D, Q, w.data());
        for (int a = 0; a < D; ++a) wee[(i * N + j) * D + a] = wee[(j * N + i) * D + a] = w[a];
      }
    std::vector<T> fnew(N * D);
    for (int i = 0; i < N; ++i) {
      // Messages, Eq. (17), normalised by the number of edges of the type.
      for (int a = 0; a < 3 * D; ++a) m[a] = T(0.0);
      for (int j = 0; j < N; ++j) {
        if (j == i) continue;
        const int t = spin(i) == spin(j) ? 0 : 1;
        for (int a = 0; a < D; ++a) m[t * D + a] += wee[(i * N + j) * D + a] * z[j * D + a];
      }
      for (int I = 0; I < M; ++I) {
        edge_embedding(s, lay, th, l, 2, den[i * M + I], e.data());
        edge_filter(th, y, 2, e.data(), D, Q, w.data());
        for (int a = 0; a < D; ++a) m[2 * D + a] += w[a] * th[y.Y + I * D + a];
      }
      const real nu[3] = {1.0 / std::max(1, n_same[spin(i)] - 1), 1.0 / std::max(1, n_opp[spin(i)]),
                            1.0 / M};
      for (int t = 0; t < 3; ++t)
        for (int a = 0; a < D; ++a) m[t * D + a] = m[t * D + a] * T(nu[t]);
      // Residual update with concatenated messages, Eq. (18), third case.
      affine(th + y.W_g, th + y.b_g, m.data(), D, 3 * D, u.data());
      for (int a = 0; a < D; ++a) fnew[i * D + a] = f[i * D + a] + tanh(u[a]);
    }
    f.swap(fnew);
  }
  if (f_out)
    for (int k = 0; k < N * D; ++k) f_out[k] = val(f[k]);

  // Orbitals x envelopes (Eqs. 8, 19, 20) and determinants: per p, either
  // det A^{up,p} det A^{down,p} (Eq. 21) or det A^p of all N electrons
  // (Eq. 22).  A determinant block covers electrons i0 .. i0 + n - 1 and n
  // orbitals; the row of electron i is filled by the orbital network and
  // envelopes of i's spin.  A_out is [blocks][K][nmax][nmax].
  const int n_blk = s.full_det ? 1 : 2;
  const int ns[2] = {s.full_det ? N : s.n_up, s.n_dn}, i0[2] = {0, s.n_up};
  const int nmax = s.full_det ? N : std::max(s.n_up, s.n_dn);
  std::vector<int> sgn_p(K, 1);
  std::vector<T> ld_p(K, T(0.0));
  for (int blk = 0; blk < n_blk; ++blk) {
    const int n = ns[blk];
    std::vector<T> phi(K * n);
    std::vector<std::vector<T>> A(K, std::vector<T>(n * n));
    for (int ii = 0; ii < n; ++ii) {
      const int i = i0[blk] + ii, sg = spin(i);
      affine(th + lay.W_o[sg], th + lay.b_o[sg], &f[i * D], K * n, D, phi.data());
      for (int p = 0; p < K; ++p)
        for (int k = 0; k < n; ++k) {
          const int o = p * n + k;
          T env(0.0);
          for (int I = 0; I < M; ++I)
            env += th[lay.omega[sg] + o * M + I] * exp(-(th[lay.zeta[sg] + o * M + I] * den[i * M + I]));
          A[p][ii * n + k] = phi[o] * env;
        }
    }
    for (int p = 0; p < K; ++p) {
      if (A_out)
        for (int ii = 0; ii < n; ++ii)
          for (int k = 0; k < n; ++k)
            A_out[((blk * K + p) * nmax + ii) * nmax + k] = val(A[p][ii * n + k]);
      int sd;
      T ld;
      slogdet(A[p], n, &sd, &ld);
      sgn_p[p] *= sd;
      ld_p[p] += ld;
    }
  }

  // Sum over determinant pairs in the log domain (Eq. 28).
  Walker<T> out;
  int pmax = -1;
  for (int p = 0; p < K; ++p) {
    const real cp = val(th[lay.c + p]);
    if (sgn_p[p] == 0 || cp == 0.0) continue;
    ld_p[p] += log(absv(th[lay.c + p]));
    if (cp < 0) sgn_p[p] = -sgn_p[p];
    if (pmax < 0 || val(ld_p[p]) > val(ld_p[pmax])) pmax = p;
  }
  if (pmax < 0) {
    out.sign = 0;
    out.logabs = T(-std::numeric_limits<real>::infinity());
    return out;
  }
  T acc(0.0);
  for (int p = 0; p < K; ++p) {
    if (sgn_p[p] == 0 || val(th[lay.c + p]) == 0.0) continue;
    T term = exp(ld_p[p] - ld_p[pmax]);
    acc += sgn_p[p] > 0 ? term : -term;
  }
  if (val(acc) == 0.0) {
    out.sign = 0;
    out.logabs = T(-std::numeric_limits<real>::infinity());
    return out;
  }
  out.sign = val(acc) > 0 ? 1 : -1;
  T logabs = ld_p[pmax] + log(absv(acc));

  // Learnable Jastrow factor J = eta(sum_i f_i^L), eta = w_J2 . tanh(W_J1 x + b_J1)  (Eq. 24).
  if (s.use_jastrow) {
    std::vector<T> sum(D, T(0.0)), h(D);
    for (int i = 0; i < N; ++i)
      for (int a = 0; a < D; ++a) sum[a] += f[i * D + a];
    affine(th + lay.W_J1, th + lay.b_J1, sum.data(), D, D, h.data());
    T J(0.0);
    for (int a = 0; a < D; ++a) J += th[lay.w_J2 + a] * tanh(h[a]);
    logabs += J;
  }
  // Electron cusp, Eq. (25): c = 1/4 same spin, 1/2 opposite spin.
  if (s.use_cusp) {
    T g(0.0);
    for (int i = 0; i < N; ++i)
      for (int j = i + 1; j < N; ++j) {
        const real c = spin(i) == spin(j) ? 0.25 : 0.5;
        g -= T(s.alpha * c) / (T(1.0) + T(s.alpha) * dee[i * N + j]);
      }
    logabs += g;
  }
  out.logabs = logabs;
  return out;
}

// Coulomb potential of Eq. (1) plus the constant nuclear repulsion.
real potential(const OracleSpec& s, const real* r) {
  const int N = s.n_up + s.n_dn, M = s.n_nuc;
  auto dist = [](const real* a, const real* b) {
    real acc = 0;
    for (int x = 0; x < 3; ++x) acc += (a[x] - b[x]) * (a[x] - b[x]);
    return std::sqrt(acc);
  };
  real V = 0;
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j) V += 1.0 / dist(r + 3 * i, r + 3 * j);
  for (int i = 0; i < N; ++i)
    for (int I = 0; I < M; ++I) V -= s.Z[I] / dist(r + 3 * i, s.R + 3 * I);
  for (int I = 0; I < M; ++I)
    for (int J = I + 1; J < M; ++J) V += s.Z[I] * s.Z[J] / dist(s.R + 3 * I, s.R + 3 * J);
  return V;
}

template <class T>
std::vector<T> lift(const real* x, int64_t n) {
  std::vector<T> y(n);
  for (int64_t k = 0; k < n; ++k) y[k] = T(x[k]);
  return y;
}

int n_threads_setting = 0;

}  // namespace

extern "C" {

int oracle_param_count(const OracleSpec* s, int64_t* P) {
  *P = Layout(*s).total;
  return 0;
}

void oracle_set_threads(int n) { n_threads_setting = n; }

int oracle_threads() {
#ifdef _OPENMP
  return n_threads_setting > 0 ? n_threads_setting : omp_get_max_threads();
#else
  return 1;
#endif
}

// log|psi|, sign psi for B walkers r[B][N][3].
int oracle_eval(const OracleSpec* s, const real* theta, const real* r, int64_t B, real* logabs,
                int8_t* sign) {
  const Layout lay(*s);
  const int N3 = 3 * (s->n_up + s->n_dn);
#pragma omp parallel for schedule(dynamic) num_threads(oracle_threads())
  for (int64_t b = 0; b < B; ++b) {
    Walker<real> w = log_psi<real>(*s, lay, theta, r + b * N3);
    logabs[b] = w.logabs;
    sign[b] = (int8_t)w.sign;
  }
  return 0;
}

// Local energy E_loc = -1/2 sum_x (d_x^2 log|psi| + (d_x log|psi|)^2) + V (Eq. 31).
// Optional grad[B][3N] and lap[B] (d_x log|psi| and sum_x d_x^2 log|psi|).
int oracle_local_energy(const OracleSpec* s, const real* theta, const real* r, int64_t B,
                        real* logabs, int8_t* sign, real* e_loc, real* grad, real* lap) {
  const Layout lay(*s);
  const int N3 = 3 * (s->n_up + s->n_dn);
  const std::vector<HD> thh = lift<HD>(theta, lay.total);
#pragma omp parallel for schedule(dynamic) num_threads(oracle_threads())
  for (int64_t b = 0; b < B; ++b) {
    const real* rb = r + b * N3;
    Walker<real> w0 = log_psi<real>(*s, lay, theta, rb);
    logabs[b] = w0.logabs;
    sign[b] = (int8_t)w0.sign;
    real sum_d2 = 0, sum_g2 = 0;
    std::vector<HD> rh = lift<HD>(rb, N3);
    for (int x = 0; x < N3; ++x) {
      rh[x].a = rh[x].b = 1.0;
      Walker<HD> w = log_psi<HD>(*s, lay, thh.data(), rh.data());
      rh[x].a = rh[x].b = 0.0;
      if (grad) grad[b * N3 + x] = w.logabs.a;
      sum_d2 += w.logabs.ab;
      sum_g2 += w.logabs.a * w.logabs.a;
    }
    if (lap) lap[b] = sum_d2;
    e_loc[b] = (w0.sign == 0 ? std::numeric_limits<real>::quiet_NaN() : -0.5 * (sum_d2 + sum_g2)) +
               potential(*s, rb);
  }
  return 0;
}

// Coulomb potential per walker.
int oracle_potential(const OracleSpec* s, const real* r, int64_t B, real* V) {
  const int N3 = 3 * (s->n_up + s->n_dn);
  for (int64_t b = 0; b < B; ++b) V[b] = potential(*s, r + b * N3);
  return 0;
}

// Directional derivatives of log|psi| in parameter space:
// out[b][k] = sum_p dirs[k][p] d log|psi_b| / d theta_p, k < n_dir.
int oracle_grad_jvp(const OracleSpec* s, const real* theta, const real* r, int64_t B,
                    const real* dirs, int32_t n_dir, real* out) {
  const Layout lay(*s);
  const int N3 = 3 * (s->n_up + s->n_dn);
  const int64_t P = lay.total;
#pragma omp parallel for collapse(2) schedule(dynamic) num_threads(oracle_threads())
  for (int64_t b = 0; b < B; ++b)
    for (int k = 0; k < n_dir; ++k) {
      std::vector<Dual> th(P);
      for (int64_t p = 0; p < P; ++p) th[p] = Dual(theta[p], dirs[(int64_t)k * P + p]);
      std::vector<Dual> rd = lift<Dual>(r + b * N3, N3);
      out[b * n_dir + k] = log_psi<Dual>(*s, lay, th.data(), rd.data()).logabs.d;
    }
  return 0;
}

// Partial derivatives d log|psi_b| / d theta_idx[k]: out[b][k].
int oracle_grad_index(const OracleSpec* s, const real* theta, const real* r, int64_t B,
                      const int64_t* idx, int32_t n_idx, real* out) {
  const Layout lay(*s);
  const int N3 = 3 * (s->n_up + s->n_dn);
  const int64_t P = lay.total;
#pragma omp parallel for collapse(2) schedule(dynamic) num_threads(oracle_threads())
  for (int64_t b = 0; b < B; ++b)
    for (int k = 0; k < n_idx; ++k) {
      std::vector<Dual> th = lift<Dual>(theta, P);
      th[idx[k]].d = 1.0;
      std::vector<Dual> rd = lift<Dual>(r + b * N3, N3);
      out[b * n_idx + k] = log_psi<Dual>(*s, lay, th.data(), rd.data()).logabs.d;
    }
  return 0;
}

// One random-walk Metropolis step (Sec. 5) on given draws:
// r' = r + step * xi;  accept iff log u < 2 (log|psi(r')| - log|psi(r)|), strict,
// and psi(r') != 0.  r[B][N][3] and logabs[B] are updated in place.
int oracle_metropolis_step(const OracleSpec* s, const real* theta, real* r, real* logabs, int64_t B,
                           const real* xi, const real* u, real step, int8_t* accepted) {
  const Layout lay(*s);
  const int N3 = 3 * (s->n_up + s->n_dn);
#pragma omp parallel for schedule(dynamic) num_threads(oracle_threads())
  for (int64_t b = 0; b < B; ++b) {
    std::vector<real> rp(N3);
    for (int x = 0; x < N3; ++x) rp[x] = r[b * N3 + x] + step * xi[b * N3 + x];
    Walker<real> w = log_psi<real>(*s, lay, theta, rp.data());
    const bool acc = w.sign != 0 && std::log(u[b]) < 2.0 * (w.logabs - logabs[b]);
    if (acc) {
      for (int x = 0; x < N3; ++x) r[b * N3 + x] = rp[x];
      logabs[b] = w.logabs;
    }
    accepted[b] = acc ? 1 : 0;
  }
  return 0;
}

// One Metropolis-adjusted Langevin step (Sec. 5, the "Langevin sampler") on
// draws passed in.  The paper names MALA with a correction that shortens the
// electron steps near the nuclei but gives no formula; this instance uses the
// drift limiting of Umrigar, Nightingale and Runge (J. Chem. Phys. 99, 2865
// (1993)) per electron with a = 1:
//   v_i = d log|psi| / d r_i,  vbar_i = v_i (sqrt(1 + 2 tau |v_i|^2) - 1) / (tau |v_i|^2),
// proposal r' = r + tau vbar(r) + sqrt(tau) xi (the Euler step of the overdamped
// Langevin dynamics whose stationary density is |psi|^2), and
//   log alpha = 2 (log|psi(r')| - log|psi(r)|) + log T(r | r') - log T(r' | r),
//   log T(y | x) = -|y - x - tau vbar(x)|^2 / (2 tau),
// accepting iff psi(r') != 0 and log u < log alpha (strict).
// grad [B][3N] holds d log|psi| / d r at r on entry and at the returned positions
// on exit (first derivatives by hyper-dual numbers, one coordinate at a time).
static void drift_limited(const real* g, int N, real tau, real* vbar) {
  for (int i = 0; i < N; ++i) {
    const real v2 = g[3 * i] * g[3 * i] + g[3 * i + 1] * g[3 * i + 1] + g[3 * i + 2] * g[3 * i + 2];
    const real s = tau * v2;
    const real f = s > 0 ? (std::sqrt(1.0 + 2.0 * s) - 1.0) / s : 1.0;
    for (int x = 0; x < 3; ++x) vbar[3 * i + x] = f * g[3 * i + x];
  }
}

int oracle_mala_step(const OracleSpec* s, const real* theta, real* r, real* logabs, real* grad, int64_t B,
                     const real* xi, const real* u, real tau, int8_t* accepted, real* log_alpha) {
  const Layout lay(*s);
  const int N = s->n_up + s->n_dn, N3 = 3 * N;
  const std::vector<HD> thh = lift<HD>(theta, lay.total);
  const real sq = std::sqrt(tau);
#pragma omp parallel for schedule(dynamic) num_threads(oracle_threads())
  for (int64_t b = 0; b < B; ++b) {
    std::vector<real> vb(N3), rp(N3), gp(N3), vbp(N3);
    drift_limited(grad + b * N3, N, tau, vb.data());
    for (int x = 0; x < N3; ++x) rp[x] = r[b * N3 + x] + tau * vb[x] + sq * xi[b * N3 + x];
    Walker<real> w = log_psi<real>(*s, lay, theta, rp.data());
    std::vector<HD> rh = lift<HD>(rp.data(), N3);
    for (int x = 0; x < N3; ++x) {
      rh[x].a = 1.0;
      gp[x] = log_psi<HD>(*s, lay, thh.data(), rh.data()).logabs.a;
      rh[x].a = 0.0;
    }
    drift_limited(gp.data(), N, tau, vbp.data());
    real fwd = 0, bwd = 0;  // |r' - r - tau vbar(r)|^2 = tau |xi|^2, and the reverse move's residual
    for (int x = 0; x < N3; ++x) {
      fwd += xi[b * N3 + x] * xi[b * N3 + x];
      const real e = r[b * N3 + x] - rp[x] - tau * vbp[x];
      bwd += e * e;
    }
    const real la = w.sign != 0 ? 2.0 * (w.logabs - logabs[b]) + 0.5 * fwd - bwd / (2.0 * tau)
                                : -std::numeric_limits<real>::infinity();
    log_alpha[b] = la;
    const bool acc = w.sign != 0 && std::log(u[b]) < la;
    if (acc) {
      for (int x = 0; x < N3; ++x) {
        r[b * N3 + x] = rp[x];
        grad[b * N3 + x] = gp[x];
      }
      logabs[b] = w.logabs;
    }
    accepted[b] = acc ? 1 : 0;
  }
  return 0;
}

// Debug views of one walker: final embeddings f[N][D] and orbital matrices
// A[2][K][nmax][nmax] (rows = electrons of the spin channel, cols = orbitals).
int oracle_intermediates(const OracleSpec* s, const real* theta, const real* r, real* f_out,
                         real* A_out) {
  const Layout lay(*s);
  log_psi<real>(*s, lay, theta, r, f_out, A_out);
  return 0;
}

}  // extern "C"
