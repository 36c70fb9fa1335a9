// Forward kernels of the ansatz with value / Jacobian / Laplacian jets.
//
// Every node quantity x of the network is carried as C channels: channel 0 is
// the value, channels 1..3N are the derivatives d x / d r_k with respect to
// the 3N electron coordinates (k = 3 i + axis), and channel C-1 is the
// Laplacian sum_k d^2 x / d r_k^2.  With C = 1 only values are computed (the
// value-only forward used by ansatz_eval and the Metropolis sampler).  Linear
// layers act on all channels alike (gemm_simt.cu); this file holds the
// nonlinear steps:
//   * geometry: distances and unit vectors of every edge and the Gaussian
//     distance features with their first two distance derivatives (Sec. 3.1);
//   * edge filters w(e(d)) as univariate jets in the distance d;
//   * graph-convolution messages (Eq. 17) with the product rule for
//     (w_ij(d_ij)) * (z_j): J(w z) = w J(z) + J(w) z and
//     L(w z) = w L(z) + L(w) z + 2 sum_k J_k(w) J_k(z), where J(w_ij) only has
//     the six coordinates of electrons i and j;
//   * the residual tanh update (Eq. 18): L(tanh u) = t' L(u) + t'' sum_k J_k(u)^2;
//   * orbitals x envelopes (Eqs. 19-20) and the determinants (Eq. 21):
//     log|det A|, d_k log|det A| = tr(A^-1 d_k A) and
//     Lap log|det A| = tr(A^-1 L(A)) - sum_k tr((A^-1 d_k A)^2), with the LU
//     factorisation in FP64 and warp-level partial pivoting;
//   * the combination over determinants (Eq. 28), the Jastrow factor (Eq. 24),
//     the electron cusp (Eq. 25), the Coulomb potential (Eq. 1) and the local
//     energy (Eq. 31).
#include <math.h>

#include "common.cuh"

namespace dq {
namespace {

constexpr int kThreads = 256;

template <class T>
__device__ __forceinline__ T tanh_t(T x) {
  return tanh(x);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Geometry and Gaussian features
// ---------------------------------------------------------------------------
template <class T>
__global__ void geometry_kernel(const T* __restrict__ r, const T* __restrict__ R, const int* __restrict__ pair_ij,
                                int64_t Bc, int N, int M, int n_ee, int E, int Q, int ej, double rc,
                                T* __restrict__ geo, T* __restrict__ rbf) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= Bc * E) return;
  const int64_t b = gid / E;
  const int e = (int)(gid % E);
  const T* rb = r + b * N * 3;
  T diff[3];
  if (e < n_ee) {
    const int i = pair_ij[2 * e], j = pair_ij[2 * e + 1];
    for (int x = 0; x < 3; ++x) diff[x] = rb[3 * i + x] - rb[3 * j + x];
  } else {
    const int i = (e - n_ee) / M, I = (e - n_ee) % M;
    for (int x = 0; x < 3; ++x) diff[x] = rb[3 * i + x] - R[3 * I + x];
  }
  const T d = sqrt(diff[0] * diff[0] + diff[1] * diff[1] + diff[2] * diff[2]);
  T* g = geo + gid * 4;
  g[0] = d;
  for (int x = 0; x < 3; ++x) g[1 + x] = diff[x] / d;
  const T s = T(rc / (Q - 1));
  const T inv_s2 = T(1) / (s * s);
  T* f = rbf + gid * ej * Q;
  for (int q = 0; q < Q; ++q) {
    const T dm = d - T(q) * s;
    const T ev = exp(T(-0.5) * dm * dm * inv_s2);
    f[q] = ev;
    if (ej == 3) {
      f[Q + q] = -dm * inv_s2 * ev;
      f[2 * Q + q] = (dm * dm * inv_s2 - T(1)) * inv_s2 * ev;
    }
  }
}

// Edge hidden layer a = tanh(W1 e + b1) as a jet in d: (a, a', a'').
template <class T>
__global__ void edge_hidden_kernel(const T* __restrict__ rbf, const T* __restrict__ params, int64_t Bc, int E,
                                   int n_par, int n_ee, int D, int Q, int ej, int64_t W1_0, int64_t W1_1,
                                   int64_t W1_2, int64_t b1_0, int64_t b1_1, int64_t b1_2, T* __restrict__ eh) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= Bc * E * D) return;
  const int a = (int)(gid % D);
  const int64_t be = gid / D;
  const int e = (int)(be % E);
  const int t = e < n_par ? 0 : (e < n_ee ? 1 : 2);
  const T* W1 = params + (t == 0 ? W1_0 : t == 1 ? W1_1 : W1_2) + (int64_t)a * Q;
  const T b1 = params[(t == 0 ? b1_0 : t == 1 ? b1_1 : b1_2) + a];
  const T* f = rbf + be * ej * Q;
  T h = b1, h1 = 0, h2 = 0;
  for (int q = 0; q < Q; ++q) {
    const T w = W1[q];
    h += w * f[q];
    if (ej == 3) {
      h1 += w * f[Q + q];
      h2 += w * f[2 * Q + q];
    }
  }
  const T av = tanh_t(h);
  T* o = eh + be * ej * D + a;
  o[0] = av;
  if (ej == 3) {
    const T da = T(1) - av * av;
    o[D] = da * h1;
    o[2 * D] = da * h2 - T(2) * av * da * h1 * h1;
  }
}

// z0[s][a] = (W_h^0 E_spin[s])[a]: the node map of layer 0 on the spin embeddings.
template <class T>
__global__ void layer0_node_kernel(const T* __restrict__ params, int D, int64_t E_spin, int64_t W_h, T* z0) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= 2 * D) return;
  const int s = gid / D, a = gid % D;
  T acc = 0;
  for (int c = 0; c < D; ++c) acc += params[W_h + (int64_t)a * D + c] * params[E_spin + s * D + c];
  z0[gid] = acc;
}

// ---------------------------------------------------------------------------
// Messages, Eq. (17), normalised per edge type, with the product rule.
// One CTA per (walker, chunk of DC features).
// ---------------------------------------------------------------------------
template <class T, int DC>
__global__ void __launch_bounds__(kThreads)
    messages_kernel(const T* __restrict__ Z, const T* __restrict__ z0, const T* __restrict__ ew,
                    const T* __restrict__ geo, const T* __restrict__ Y, const int* __restrict__ pair_of, int N,
                    int n_up, int M, int C, int D, int E, int n_ee, int ej, int z_const, T* __restrict__ msg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Zs = reinterpret_cast<T*>(smem_raw);                 // [N][C][DC] (or [2][DC] if z_const)
  const int zs_elems = z_const ? 2 * DC : N * C * DC;
  T* EWs = Zs + zs_elems;                                 // [E][ej][DC]
  T* Ys = EWs + (int64_t)E * ej * DC;                     // [M][DC]
  T* Gs = Ys + M * DC;                                    // [E][4]
  int* Ps = reinterpret_cast<int*>(Gs + E * 4);           // [N][N]

  const int64_t b = blockIdx.x;
  const int d0 = blockIdx.y * DC;
  const int tid = threadIdx.x;

  if (z_const) {
    for (int k = tid; k < 2 * DC; k += kThreads) Zs[k] = z0[(k / DC) * D + d0 + k % DC];
  } else {
    const T* Zb = Z + b * N * C * D;
    for (int k = tid; k < N * C * DC; k += kThreads) Zs[k] = Zb[(int64_t)(k / DC) * D + d0 + k % DC];
  }
  const T* EWb = ew + b * E * ej * D;
  for (int k = tid; k < E * ej * DC; k += kThreads) EWs[k] = EWb[(int64_t)(k / DC) * D + d0 + k % DC];
  for (int k = tid; k < M * DC; k += kThreads) Ys[k] = Y[(int64_t)(k / DC) * D + d0 + k % DC];
  const T* Gb = geo + b * E * 4;
  for (int k = tid; k < E * 4; k += kThreads) Gs[k] = Gb[k];
  for (int k = tid; k < N * N; k += kThreads) Ps[k] = pair_of[k];
  __syncthreads();

  const int n_dn = N - n_up;
  const bool jets = C > 1;
  const int dd = tid % DC;
  const int ngroups = kThreads / DC;
  auto zval = [&](int j, int c) -> T {
    if (z_const) return c == 0 ? Zs[(j < n_up ? 0 : 1) * DC + dd] : T(0);
    return Zs[(j * C + c) * DC + dd];
  };
  T* mb = msg + b * N * C * 3 * D;
  for (int oc = tid / DC; oc < N * C; oc += ngroups) {
    const int i = oc / C, c = oc % C;
    const bool up_i = i < n_up;
    const bool isJ = jets && c >= 1 && c < C - 1;
    const bool isL = jets && c == C - 1;
    const int ke = isJ ? (c - 1) / 3 : -1, kx = isJ ? (c - 1) % 3 : 0;
    T acc_s = 0, acc_o = 0, acc_n = 0;
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      const int p = Ps[i * N + j];
      const T sg = i < j ? T(1) : T(-1);  // unit vectors are stored for (min, max)
      const T w = EWs[(p * ej) * DC + dd];
      T v = w * zval(j, c);
      if (isJ && (ke == i || ke == j)) {
        const T t = EWs[(p * ej + 1) * DC + dd] * sg * Gs[p * 4 + 1 + kx] * zval(j, 0);
        v += ke == i ? t : -t;
      }
      if (isL) {
        const T w1 = EWs[(p * ej + 1) * DC + dd], w2 = EWs[(p * ej + 2) * DC + dd];
        v += (T(2) * w2 + T(4) * w1 / Gs[p * 4]) * zval(j, 0);
        T s = 0;
        for (int x = 0; x < 3; ++x) s += sg * Gs[p * 4 + 1 + x] * (zval(j, 1 + 3 * i + x) - zval(j, 1 + 3 * j + x));
        v += T(2) * w1 * s;
      }
      if ((j < n_up) == up_i)
        acc_s += v;
      else
        acc_o += v;
    }
    for (int I = 0; I < M; ++I) {
      const int e = n_ee + i * M + I;
      const T y = Ys[I * DC + dd];
      if (c == 0) acc_n += EWs[(e * ej) * DC + dd] * y;
      if (isJ && ke == i) acc_n += EWs[(e * ej + 1) * DC + dd] * Gs[e * 4 + 1 + kx] * y;
      if (isL) acc_n += (EWs[(e * ej + 2) * DC + dd] + T(2) * EWs[(e * ej + 1) * DC + dd] / Gs[e * 4]) * y;
    }
    const int n_same = up_i ? n_up : n_dn, n_opp = up_i ? n_dn : n_up;
    const T nu_s = T(1) / T(n_same - 1 > 1 ? n_same - 1 : 1);
    const T nu_o = T(1) / T(n_opp > 1 ? n_opp : 1);
    const T nu_n = T(1) / T(M);
    T* o = mb + ((int64_t)i * C + c) * 3 * D + d0 + dd;
    o[0] = acc_s * nu_s;
    o[D] = acc_o * nu_o;
    o[2 * D] = acc_n * nu_n;
  }
}

// ---------------------------------------------------------------------------
// Residual tanh update, Eq. (18): f <- f + tanh(P) with jets.
// ---------------------------------------------------------------------------
template <class T>
__global__ void update_kernel(const T* __restrict__ P, T* __restrict__ F, const T* __restrict__ E_spin,
                              int64_t Bc, int N, int n_up, int C, int D, int from_spin) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= Bc * N * D) return;
  const int a = (int)(gid % D);
  const int64_t bi = gid / D;
  const int i = (int)(bi % N);
  const T* p = P + bi * C * D + a;
  T* f = F + bi * C * D + a;
  const T t = tanh_t(p[0]);
  const T dt = T(1) - t * t;
  f[0] = (from_spin ? E_spin[(i < n_up ? 0 : 1) * D + a] : f[0]) + t;
  if (C > 1) {
    T ss = 0;
    for (int c = 1; c < C - 1; ++c) {
      const T pc = p[(int64_t)c * D];
      ss += pc * pc;
      f[(int64_t)c * D] = (from_spin ? T(0) : f[(int64_t)c * D]) + dt * pc;
    }
    const int64_t cl = (int64_t)(C - 1) * D;
    f[cl] = (from_spin ? T(0) : f[cl]) + dt * p[cl] - T(2) * t * dt * ss;
  }
}

// ---------------------------------------------------------------------------
// Orbitals x envelopes and determinant jets.  One warp per (walker, spin, p).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(128)
    orbital_det_kernel(const T* __restrict__ phi, const T* __restrict__ geo, const T* __restrict__ params,
                       int64_t Bc, int N, int n_up, int M, int K, int C, int Wo, int E, int n_ee,
                       int64_t om_up, int64_t om_dn, int64_t ze_up, int64_t ze_dn, double* __restrict__ det) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int warps = blockDim.x / 32;
  const int64_t gw = (int64_t)blockIdx.x * warps + warp;
  const int n_dn = N - n_up;
  const int nmax = n_up > n_dn ? n_up : n_dn;
  const int N3 = 3 * N;
  const bool jets = C > 1;
  // per-warp shared memory
  const int nn = nmax * nmax;
  const size_t per_warp = (size_t)nn * (3 * sizeof(double) + 7 * sizeof(T)) + 32 * sizeof(int);
  unsigned char* base = smem_raw + warp * ((per_warp + 15) / 16 * 16);
  double* LU = reinterpret_cast<double*>(base);
  double* Ainv = LU + nn;
  T* env = reinterpret_cast<T*>(Ainv + 2 * nn);
  T* jenv = env + nn;      // [3][nn]
  T* lenv = jenv + 3 * nn;
  T* phi0 = lenv + nn;
  T* tmp = phi0 + nn;      // one tangent of A
  double* X = reinterpret_cast<double*>(base) + 2 * nn;  // A^-1 d_k A (FP64)
  int* perm = reinterpret_cast<int*>(tmp + nn);

  if (gw >= Bc * 2 * K) return;
  const int64_t b = gw / (2 * K);
  const int s = (int)((gw / K) % 2);
  const int p = (int)(gw % K);
  const int n = s == 0 ? n_up : n_dn;
  const int i0 = s == 0 ? 0 : n_up;
  double* out = det + gw * (N3 + 3);
  if (n == 0) {  // empty determinant = 1
    for (int k = lane; k < N3 + 3; k += 32) out[k] = k == 0 ? 1.0 : 0.0;
    return;
  }
  const T* om = params + (s == 0 ? om_up : om_dn);
  const T* ze = params + (s == 0 ? ze_up : ze_dn);
  const T* phib = phi + b * N * C * Wo;
  const T* gb = geo + b * E * 4;

  // Envelopes (Eq. 20) with their derivatives in the coordinates of electron i.
  for (int q = lane; q < n * n; q += 32) {
    const int ii = q / n, k = q % n, o = p * n + k, i = i0 + ii;
    T ev = 0, j0 = 0, j1 = 0, j2 = 0, lv = 0;
    for (int I = 0; I < M; ++I) {
      const T* g = gb + (n_ee + i * M + I) * 4;
      const T z = ze[o * M + I];
      const T w = om[o * M + I] * exp(-z * g[0]);
      ev += w;
      j0 -= w * z * g[1];
      j1 -= w * z * g[2];
      j2 -= w * z * g[3];
      lv += w * (z * z - T(2) * z / g[0]);
    }
    env[q] = ev;
    jenv[q] = j0;
    jenv[nn + q] = j1;
    jenv[2 * nn + q] = j2;
    lenv[q] = lv;
    const T f0 = phib[(int64_t)i * C * Wo + o];
    phi0[q] = f0;
    LU[q] = (double)f0 * (double)ev;
  }
  if (lane < n) perm[lane] = lane;
  __syncwarp();

  // LU with partial pivoting (FP64), pivot search across the warp.
  int sign = 1;
  double logabs = 0.0;
  bool singular = false;
  for (int j = 0; j < n; ++j) {
    double v = (lane >= j && lane < n) ? fabs(LU[lane * n + j]) : -1.0;
    int idx = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
      if (v2 > v || (v2 == v && i2 < idx)) {
        v = v2;
        idx = i2;
      }
    }
    if (!(v > 0.0)) {
      singular = true;
      break;
    }
    if (idx != j) {
      for (int k = lane; k < n; k += 32) {
        const double t = LU[j * n + k];
        LU[j * n + k] = LU[idx * n + k];
        LU[idx * n + k] = t;
      }
      if (lane == 0) {
        const int t = perm[j];
        perm[j] = perm[idx];
        perm[idx] = t;
      }
      sign = -sign;
    }
    __syncwarp();
    const double piv = LU[j * n + j];
    for (int i = j + 1 + lane; i < n; i += 32) {
      const double f = LU[i * n + j] / piv;
      LU[i * n + j] = f;
      for (int k = j + 1; k < n; ++k) LU[i * n + k] -= f * LU[j * n + k];
    }
    __syncwarp();
    if (piv < 0) sign = -sign;
    logabs += log(fabs(piv));
  }
  if (singular) {
    for (int k = lane; k < N3 + 3; k += 32) out[k] = k == 1 ? -INFINITY : 0.0;
    return;
  }
  if (lane == 0) {
    out[0] = (double)sign;
    out[1] = logabs;
  }
  if (!jets) return;

  // A^-1 column by column: lane solves L U x = P e_col.
  if (lane < n) {
    const int col = lane;
    double* x = Ainv;  // stored as Ainv[row][col]
    for (int r = 0; r < n; ++r) {
      double acc = perm[r] == col ? 1.0 : 0.0;
      for (int m = 0; m < r; ++m) acc -= LU[r * n + m] * x[m * n + col];
      x[r * n + col] = acc;
    }
    for (int r = n - 1; r >= 0; --r) {
      double acc = x[r * n + col];
      for (int m = r + 1; m < n; ++m) acc -= LU[r * n + m] * x[m * n + col];
      x[r * n + col] = acc / LU[r * n + r];
    }
  }
  __syncwarp();

  // Tangents: d_k A = d_k phi * env + phi * d_k env (env depends on electron i only).
  // LU, A^-1, log|det| and the tangent contractions are FP64.
  double lap = 0.0;
  for (int t = 0; t <= N3; ++t) {
    const bool is_lap = t == N3;
    const int c = is_lap ? C - 1 : 1 + t;
    for (int q = lane; q < n * n; q += 32) {
      const int ii = q / n, k = q % n, o = p * n + k, i = i0 + ii;
      const T* ph = phib + (int64_t)i * C * Wo + o;
      T v = ph[(int64_t)c * Wo] * env[q];
      if (is_lap) {
        v += phi0[q] * lenv[q];
        for (int x = 0; x < 3; ++x) v += T(2) * ph[(int64_t)(1 + 3 * i + x) * Wo] * jenv[x * nn + q];
      } else if (t / 3 == i) {
        v += phi0[q] * jenv[(t % 3) * nn + q];
      }
      tmp[q] = v;
    }
    __syncwarp();
    // X = A^-1 dA; tr X = d log|det A|
    double trp = 0;
    for (int q = lane; q < n * n; q += 32) {
      const int a = q / n, m = q % n;
      double x = 0;
      for (int l = 0; l < n; ++l) x += Ainv[a * n + l] * (double)tmp[l * n + m];
      X[q] = x;
      if (a == m) trp += x;
    }
    const double tr = warp_sum(trp);
    __syncwarp();
    if (is_lap) {
      lap += tr;
    } else {
      if (lane == 0) out[2 + t] = tr;
      // tr(X^2) = sum_{a,m} X[a][m] X[m][a]
      double s2 = 0;
      for (int q = lane; q < n * n; q += 32) {
        const int a = q / n, m = q % n;
        s2 += X[a * n + m] * X[m * n + a];
      }
      lap -= warp_sum(s2);
    }
    __syncwarp();
  }
  if (lane == 0) out[2 + N3] = lap;
}

// Sum of embeddings over electrons, the input of the Jastrow factor (Eq. 24).
template <class T>
__global__ void jastrow_sum_kernel(const T* __restrict__ F, int64_t Bc, int N, int C, int D, T* __restrict__ js) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= Bc * C * D) return;
  const int64_t b = gid / (C * D);
  const int64_t cd = gid % (C * D);
  T acc = 0;
  for (int i = 0; i < N; ++i) acc += F[(b * N + i) * C * D + cd];
  js[gid] = acc;
}

// ---------------------------------------------------------------------------
// Combination over determinants, Jastrow, cusp, potential and E_loc.
// One CTA per walker; all arithmetic in FP64.
// ---------------------------------------------------------------------------
constexpr int kCombineThreads = 128;

__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kCombineThreads / 32 ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

template <class T>
__global__ void __launch_bounds__(kCombineThreads)
    combine_kernel(const double* __restrict__ det, const T* __restrict__ jh, const T* __restrict__ geo,
                   const T* __restrict__ params, const double* __restrict__ Zn, const int* __restrict__ pair_ij,
                   const int* __restrict__ pair_of, int64_t Bc, int N, int n_up, int M, int K, int C, int D, int E, int n_ee, int64_t c_off,
                   int64_t wJ2_off, int use_jastrow, int use_cusp, double alpha, double Vnn, T* __restrict__ logabs,
                   int8_t* __restrict__ sign_out, T* __restrict__ e_loc, unsigned int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N3 = 3 * N;
  double* wp = reinterpret_cast<double*>(smem_raw);  // [K] determinant weights
  double* gsq = wp + K;                              // [K] |grad l_p|^2
  double* td = gsq + K;                              // [3][D] Jastrow: w t, w t', w t''
  double* red = td + 3 * D;                          // [32]
  __shared__ double s_scalar[4];
  const int64_t b = blockIdx.x;
  const int tid = threadIdx.x;
  const bool jets = C > 1;
  const double* db = det + b * 2 * K * (N3 + 3);
  auto dp = [&](int s, int p) { return db + ((int64_t)s * K + p) * (N3 + 3); };

  // log-sum-exp over determinant pairs (Eq. 28)
  if (tid == 0) {
    double lmax = -INFINITY;
    for (int p = 0; p < K; ++p) {
      const double cp = (double)params[c_off + p];
      const double sp = dp(0, p)[0] * dp(1, p)[0] * (cp > 0 ? 1.0 : cp < 0 ? -1.0 : 0.0);
      const double lp = sp != 0.0 ? dp(0, p)[1] + dp(1, p)[1] + log(fabs(cp)) : -INFINITY;
      wp[p] = lp;
      gsq[p] = sp;
      if (sp != 0.0 && lp > lmax) lmax = lp;
    }
    double S = 0.0;
    if (lmax > -INFINITY)
      for (int p = 0; p < K; ++p)
        if (gsq[p] != 0.0) S += gsq[p] * exp(wp[p] - lmax);
    for (int p = 0; p < K; ++p) wp[p] = (gsq[p] != 0.0 && S != 0.0) ? gsq[p] * exp(wp[p] - lmax) / S : 0.0;
    s_scalar[0] = S > 0 ? 1.0 : (S < 0 ? -1.0 : 0.0);
    s_scalar[1] = S != 0.0 ? lmax + log(fabs(S)) : -INFINITY;
  }
  __syncthreads();
  const double sgn = s_scalar[0];
  double la = s_scalar[1];

  // Jastrow factor values and tanh derivatives per feature
  const T* jb = jh + b * C * D;
  double Jv = 0.0;
  if (use_jastrow) {
    double part = 0.0;
    for (int a = tid; a < D; a += kCombineThreads) {
      const double w = (double)params[wJ2_off + a];
      const double t = tanh((double)jb[a]);
      const double dt = 1.0 - t * t;
      td[a] = w * t;
      td[D + a] = w * dt;
      td[2 * D + a] = -2.0 * w * t * dt;
      part += w * t;
    }
    Jv = block_sum(part, red);
  }
  // cusp value and potential
  const T* gb = geo + b * E * 4;
  double gpart = 0.0, vpart = 0.0;
  for (int e = tid; e < n_ee; e += kCombineThreads) {
    const double d = (double)gb[e * 4];
    vpart += 1.0 / d;
    if (use_cusp) {
      const int i = pair_ij[2 * e], j = pair_ij[2 * e + 1];
      const double c = ((i < n_up) == (j < n_up)) ? 0.25 : 0.5;
      gpart -= alpha * c / (1.0 + alpha * d);
    }
  }
  for (int e = n_ee + tid; e < E; e += kCombineThreads) vpart -= Zn[(e - n_ee) % M] / (double)gb[e * 4];
  const double gam = use_cusp ? block_sum(gpart, red) : 0.0;
  const double V = block_sum(vpart, red) + Vnn;
  la += Jv + gam;

  if (!jets) {
    if (tid == 0) {
      logabs[b] = sgn != 0.0 ? (T)la : (T)(-INFINITY);
      sign_out[b] = (int8_t)sgn;
      if (sgn == 0.0) atomicOr(status, (unsigned)DQ_FLAG_SINGULAR);
    }
    return;
  }
  // |grad l_p|^2 per determinant pair
  for (int p = tid; p < K; p += kCombineThreads) {
    double acc = 0.0;
    for (int k = 0; k < N3; ++k) {
      const double g = dp(0, p)[2 + k] + dp(1, p)[2 + k];
      acc += g * g;
    }
    gsq[p] = acc;
  }
  __syncthreads();
  // gradient components and the Jastrow Laplacian term
  double g2part = 0.0, lJpart = 0.0;
  for (int k = tid; k < N3; k += kCombineThreads) {
    double g = 0.0;
    for (int p = 0; p < K; ++p) g += wp[p] * (dp(0, p)[2 + k] + dp(1, p)[2 + k]);
    if (use_jastrow) {
      const T* row = jb + (int64_t)(1 + k) * D;
      double gj = 0.0, lj = 0.0;
      for (int a = 0; a < D; ++a) {
        const double h = (double)row[a];
        gj += td[D + a] * h;
        lj += td[2 * D + a] * h * h;
      }
      g += gj;
      lJpart += lj;
    }
    if (use_cusp) {
      const int e = k / 3, x = k % 3;
      for (int j = 0; j < N; ++j) {
        if (j == e) continue;
        const int pidx = pair_of[e * N + j];
        const double d = (double)gb[pidx * 4];
        const double u = (double)gb[pidx * 4 + 1 + x] * (e < j ? 1.0 : -1.0);
        const double c = ((e < n_up) == (j < n_up)) ? 0.25 : 0.5;
        const double q1 = 1.0 + alpha * d;
        g += alpha * alpha * c / (q1 * q1) * u;
      }
    }
    g2part += g * g;
  }
  // Laplacian terms
  double lpart = lJpart;
  for (int p = tid; p < K; p += kCombineThreads) lpart += wp[p] * (dp(0, p)[2 + N3] + dp(1, p)[2 + N3] + gsq[p]);
  if (use_jastrow)
    for (int a = tid; a < D; a += kCombineThreads) lpart += td[D + a] * (double)jb[(int64_t)(C - 1) * D + a];
  if (use_cusp)
    for (int e = tid; e < n_ee; e += kCombineThreads) {
      const int i = pair_ij[2 * e], j = pair_ij[2 * e + 1];
      const double c = ((i < n_up) == (j < n_up)) ? 0.25 : 0.5;
      const double d = (double)gb[e * 4];
      const double q1 = 1.0 + alpha * d;
      const double g1 = alpha * alpha * c / (q1 * q1);
      const double g2 = -2.0 * alpha * alpha * alpha * c / (q1 * q1 * q1);
      lpart += 2.0 * g2 + 4.0 * g1 / d;
    }
  // squared gradient of the determinant part enters with a minus sign:
  // Lap log|psi_D| = sum_p w_p (Lap l_p + |grad l_p|^2) - |grad log|psi_D||^2
  double gD2part = 0.0;
  for (int k = tid; k < N3; k += kCombineThreads) {
    double g = 0.0;
    for (int p = 0; p < K; ++p) g += wp[p] * (dp(0, p)[2 + k] + dp(1, p)[2 + k]);
    gD2part += g * g;
  }
  const double g2 = block_sum(g2part, red);
  const double lap = block_sum(lpart, red) - block_sum(gD2part, red);
  if (tid == 0) {
    double el = -0.5 * (lap + g2) + V;
    logabs[b] = sgn != 0.0 ? (T)la : (T)(-INFINITY);
    sign_out[b] = (int8_t)sgn;
    if (sgn == 0.0) {
      el = NAN;
      atomicOr(status, (unsigned)DQ_FLAG_SINGULAR);
    }
    if (!isfinite(el)) atomicOr(status, (unsigned)DQ_FLAG_NONFINITE);
    e_loc[b] = (T)el;
  }
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <class T>
cudaError_t launch_geometry(const dq_handle_s& h, const FwdDims& d, const T* r, FwdBuffers<T> b, cudaStream_t s) {
  const T* R = nullptr;
  if constexpr (sizeof(T) == 8) R = h.d_R; else R = h.d_Rf;
  const int ej = d.C > 1 ? 3 : 1;
  geometry_kernel<T><<<blocks(d.Bc * h.edges.n_all, 128), 128, 0, s>>>(
      r, R, h.d_pair_ij, d.Bc, d.N, d.M, h.edges.n_ee, h.edges.n_all, d.Q, ej, h.rc, b.geo, b.rbf);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_edge_hidden(const dq_handle_s& h, const FwdDims& d, const T* params, int l, FwdBuffers<T> b,
                               cudaStream_t s) {
  const int ej = d.C > 1 ? 3 : 1;
  const auto& y = h.off.layer[l];
  const int64_t n = d.Bc * h.edges.n_all * d.D;
  edge_hidden_kernel<T><<<blocks(n, 256), 256, 0, s>>>(b.rbf, params, d.Bc, h.edges.n_all, h.edges.n_par,
                                                       h.edges.n_ee, d.D, d.Q, ej, y.W1[0], y.W1[1], y.W1[2],
                                                       y.b1[0], y.b1[1], y.b1[2], b.eh);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_layer0_node(const dq_handle_s& h, const FwdDims& d, const T* params, FwdBuffers<T> b,
                               cudaStream_t s) {
  layer0_node_kernel<T><<<blocks(2 * d.D, 128), 128, 0, s>>>(params, d.D, h.off.E_spin, h.off.layer[0].W_h, b.z0);
  return cudaGetLastError();
}

namespace {
template <class T>
size_t message_smem(const dq_handle_s& h, const FwdDims& d, int DC, bool z_const) {
  const int ej = d.C > 1 ? 3 : 1;
  const int E = h.edges.n_all;
  const size_t zs = z_const ? 2 * DC : (size_t)d.N * d.C * DC;
  return (zs + (size_t)E * ej * DC + (size_t)d.M * DC + (size_t)E * 4) * sizeof(T) + (size_t)d.N * d.N * sizeof(int);
}
template <class T, int DC>
cudaError_t launch_messages_dc(const dq_handle_s& h, const FwdDims& d, const T* params, int l, bool z_const,
                               FwdBuffers<T> b, size_t smem, cudaStream_t s) {
  auto kern = messages_kernel<T, DC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)d.Bc, d.D / DC);
  kern<<<grid, kThreads, smem, s>>>(b.Z, b.z0, b.ew, b.geo, params + h.off.layer[l].Y, h.d_pair_of, d.N, d.n_up, d.M,
                                    d.C, d.D, h.edges.n_all, h.edges.n_ee, d.C > 1 ? 3 : 1, z_const ? 1 : 0, b.msg);
  return cudaGetLastError();
}
}  // namespace

template <class T>
cudaError_t launch_messages(const dq_handle_s& h, const FwdDims& d, const T* params, int l, bool z_const,
                            FwdBuffers<T> b, cudaStream_t s) {
  constexpr size_t kBudget = 96 * 1024, kMax = 220 * 1024;
  for (int DC : {32, 16, 8, 4}) {
    if (d.D % DC) continue;
    const size_t smem = message_smem<T>(h, d, DC, z_const);
    if (smem > kBudget && DC > 4) continue;
    if (smem > kMax) return cudaErrorInvalidConfiguration;
    switch (DC) {
      case 32: return launch_messages_dc<T, 32>(h, d, params, l, z_const, b, smem, s);
      case 16: return launch_messages_dc<T, 16>(h, d, params, l, z_const, b, smem, s);
      case 8: return launch_messages_dc<T, 8>(h, d, params, l, z_const, b, smem, s);
      default: return launch_messages_dc<T, 4>(h, d, params, l, z_const, b, smem, s);
    }
  }
  return cudaErrorInvalidConfiguration;
}

template <class T>
cudaError_t launch_update(const dq_handle_s& h, const FwdDims& d, const T* params, bool from_spin, FwdBuffers<T> b,
                          cudaStream_t s) {
  update_kernel<T><<<blocks(d.Bc * d.N * d.D, 256), 256, 0, s>>>(b.Z, b.F, params + h.off.E_spin, d.Bc, d.N, d.n_up,
                                                                 d.C, d.D, from_spin ? 1 : 0);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_orbital_det(const dq_handle_s& h, const FwdDims& d, const T* params, FwdBuffers<T> b,
                               cudaStream_t s) {
  const int nmax = d.n_up > d.n_dn ? d.n_up : d.n_dn;
  const int nn = nmax * nmax;
  const size_t per_warp = ((size_t)nn * (3 * sizeof(double) + 7 * sizeof(T)) + 32 * sizeof(int) + 15) / 16 * 16;
  const int warps = 4;
  const size_t smem = per_warp * warps;
  auto kern = orbital_det_kernel<T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t nmat = d.Bc * 2 * d.K;
  kern<<<blocks(nmat, warps), warps * 32, smem, s>>>(b.phi, b.geo, params, d.Bc, d.N, d.n_up, d.M, d.K, d.C,
                                                     d.K * nmax, h.edges.n_all, h.edges.n_ee, h.off.omega[0],
                                                     h.off.omega[1], h.off.zeta[0], h.off.zeta[1], b.det);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_jastrow_sum(const dq_handle_s& h, const FwdDims& d, FwdBuffers<T> b, cudaStream_t s) {
  (void)h;
  jastrow_sum_kernel<T><<<blocks(d.Bc * d.C * d.D, 256), 256, 0, s>>>(b.F, d.Bc, d.N, d.C, d.D, b.js);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_combine(const dq_handle_s& h, const FwdDims& d, const T* params, FwdBuffers<T> b, T* logabs,
                           int8_t* sign, T* e_loc, cudaStream_t s) {
  const size_t smem = (2 * (size_t)d.K + 3 * (size_t)d.D + 32) * sizeof(double);
  auto kern = combine_kernel<T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)d.Bc, kCombineThreads, smem, s>>>(
      b.det, b.jh, b.geo, params, h.d_Z, h.d_pair_ij, h.d_pair_of, d.Bc, d.N, d.n_up, d.M, d.K, d.C, d.D, h.edges.n_all,
      h.edges.n_ee, h.off.c, h.off.w_J2, h.use_jastrow, h.use_cusp, h.alpha, h.Vnn, logabs, sign, e_loc, h.d_status);
  return cudaGetLastError();
}

#define DQ_INSTANTIATE(T)                                                                                          \
  template cudaError_t launch_geometry<T>(const dq_handle_s&, const FwdDims&, const T*, FwdBuffers<T>,            \
                                          cudaStream_t);                                                          \
  template cudaError_t launch_edge_hidden<T>(const dq_handle_s&, const FwdDims&, const T*, int, FwdBuffers<T>,    \
                                             cudaStream_t);                                                       \
  template cudaError_t launch_layer0_node<T>(const dq_handle_s&, const FwdDims&, const T*, FwdBuffers<T>,         \
                                             cudaStream_t);                                                       \
  template cudaError_t launch_messages<T>(const dq_handle_s&, const FwdDims&, const T*, int, bool, FwdBuffers<T>, \
                                          cudaStream_t);                                                          \
  template cudaError_t launch_update<T>(const dq_handle_s&, const FwdDims&, const T*, bool, FwdBuffers<T>,        \
                                        cudaStream_t);                                                            \
  template cudaError_t launch_orbital_det<T>(const dq_handle_s&, const FwdDims&, const T*, FwdBuffers<T>,         \
                                             cudaStream_t);                                                       \
  template cudaError_t launch_jastrow_sum<T>(const dq_handle_s&, const FwdDims&, FwdBuffers<T>, cudaStream_t);    \
  template cudaError_t launch_combine<T>(const dq_handle_s&, const FwdDims&, const T*, FwdBuffers<T>, T*,         \
                                         int8_t*, T*, cudaStream_t);

DQ_INSTANTIATE(float)
DQ_INSTANTIATE(double)

}  // namespace dq
