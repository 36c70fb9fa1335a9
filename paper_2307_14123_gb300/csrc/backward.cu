// Reverse pass of the value-only network: d log|psi| / d theta (Sec. 4.1,
// Eq. 30 needs grad_theta log|psi| per walker).
//
// The seed of walker b is its weight w_b (weighted mode) or 1 (per-walker
// mode); walkers with psi = 0 get seed 0.  Adjoints flow backwards through
//   log|psi| = log|sum_p c_p det A_up^p det A_dn^p| + J + gamma   (Eqs. 21, 24, 25, 28)
// with d log|psi_D| / d log|det A^{s,p}| = w_p (the signed weight of pair p in
// the log-sum-exp) and d log|det A| / d A = A^-T; then through the orbital
// head and envelopes (Eqs. 19-20), and per layer through the residual tanh
// update (Eq. 18), the graph-convolution messages (Eq. 17), the node map and
// the edge filters.  Parameter gradients are sums over rows (electrons, edges
// or walkers) of products of an adjoint and a saved activation; they are
// formed by param_reduce, per walker or summed over walkers.
#include <math.h>

#include <algorithm>

#include "backward.cuh"
#include "det_util.cuh"

namespace dq {
namespace {

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Combination over determinant pairs and Jastrow factor.  One warp per walker.
//   beta[b][p]  = g_b w_p      (adjoint of log|det A^{s,p}|, both spins)
//   cbar[b][p]  = g_b q_p,     q_p = det A_up^p det A_dn^p / psi_D
//   jhbar[b][a] = g_b w_J2[a] (1 - t_a^2),  t = tanh(W_J1 s + b_J1)
//   gt[b][a]    = g_b t_a      (adjoint of w_J2)
// ---------------------------------------------------------------------------
template <class T>
__global__ void bwd_combine_kernel(const double* __restrict__ det, const T* __restrict__ jh,
                                   const T* __restrict__ params, const T* __restrict__ weights, int64_t Bc, int N,
                                   int K, int D, int64_t c_off, int64_t wJ2_off, int use_jastrow,
                                   T* __restrict__ beta, T* __restrict__ cbar, T* __restrict__ jhbar,
                                   T* __restrict__ gt) {
  const int lane = threadIdx.x % 32;
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  if (b >= Bc) return;
  const int N3 = 3 * N;
  const double* db = det + b * 2 * K * (N3 + 3);
  auto dp = [&](int s, int p) { return db + ((int64_t)s * K + p) * (N3 + 3); };
  // lmax and the signed sum (same reduction as the forward combine)
  double lmax = -INFINITY;
  for (int p = lane; p < K; p += 32) {
    const double cp = (double)params[c_off + p];
    const double sp = dp(0, p)[0] * dp(1, p)[0] * (cp > 0 ? 1.0 : cp < 0 ? -1.0 : 0.0);
    if (sp != 0.0) lmax = fmax(lmax, dp(0, p)[1] + dp(1, p)[1] + log(fabs(cp)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  double S = 0.0;
  if (lmax > -INFINITY)
    for (int p = lane; p < K; p += 32) {
      const double cp = (double)params[c_off + p];
      const double sp = dp(0, p)[0] * dp(1, p)[0] * (cp > 0 ? 1.0 : cp < 0 ? -1.0 : 0.0);
      if (sp != 0.0) S += sp * exp(dp(0, p)[1] + dp(1, p)[1] + log(fabs(cp)) - lmax);
    }
  S = warp_sum_d(S);
  double g = weights ? (double)weights[b] : 1.0;
  if (!(S != 0.0) || !isfinite(S)) g = 0.0;  // psi = 0: no gradient
  for (int p = lane; p < K; p += 32) {
    const double s2 = dp(0, p)[0] * dp(1, p)[0];
    double q = 0.0;
    if (g != 0.0 && s2 != 0.0) q = s2 * exp(dp(0, p)[1] + dp(1, p)[1] - lmax) / S;
    const double cp = (double)params[c_off + p];
    cbar[b * K + p] = (T)(g * q);
    beta[b * K + p] = (T)(g * q * cp);
  }
  for (int a = lane; a < D; a += 32) {
    double jb = 0.0, tt = 0.0;
    if (use_jastrow) {
      const double t = tanh((double)jh[b * D + a]);
      jb = g * (double)params[wJ2_off + a] * (1.0 - t * t);
      tt = g * t;
    }
    jhbar[b * D + a] = (T)jb;
    gt[b * D + a] = (T)tt;
  }
}

// ---------------------------------------------------------------------------
// Determinants and envelopes.  One warp per (walker, spin, p).
//   Abar = beta_p A^-T;  phibar_ik = Abar_ik env_ik;  envbar_ik = Abar_ik phi_ik
//   omegabar_oI = sum_i envbar_ik exp(-zeta_oI d_iI)
//   zetabar_oI  = sum_i envbar_ik omega_oI (-d_iI) exp(-zeta_oI d_iI)
// A^-1 from an LU in the arithmetic type; in FP32 modes near-nodal matrices
// (row-equilibrated condition estimate above 1000) are redone in FP64.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(128)
    bwd_det_kernel(const T* __restrict__ phi, const T* __restrict__ geo, const T* __restrict__ params,
                   const T* __restrict__ beta, int64_t Bc, int N, int n_up, int M, int K, int Wo, int E, int n_ee,
                   int64_t om_up, int64_t om_dn, int64_t ze_up, int64_t ze_dn, T* __restrict__ phibar,
                   T* __restrict__ envbar, int full) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int warps = blockDim.x / 32;
  const int64_t gw = (int64_t)blockIdx.x * warps + warp;
  const int n_dn = N - n_up;
  const int nmax = full ? N : (n_up > n_dn ? n_up : n_dn);
  const int nn = nmax * nmax;
  const size_t per_warp = (size_t)nn * (2 * sizeof(double) + 5 * sizeof(T)) + 32 * sizeof(int);
  unsigned char* base = smem_raw + warp * ((per_warp + 15) / 16 * 16);
  double* LUd = reinterpret_cast<double*>(base);
  double* Ainvd = LUd + nn;
  T* env = reinterpret_cast<T*>(Ainvd + nn);
  T* phi0 = env + nn;
  T* LUt = phi0 + nn;
  T* Ainvt = LUt + nn;
  T* rmax = Ainvt + nn;
  int* perm = reinterpret_cast<int*>(rmax + nn);
  if (gw >= Bc * 2 * K) return;
  const int64_t b = gw / (2 * K);
  const int s = (int)((gw / K) % 2);
  const int p = (int)(gw % K);
  // Block s: the spin-s matrix of Eq. (21), or (full) the N x N matrix of
  // Eq. (22) for s = 0 and nothing for s = 1.  Row ii is electron i0 + ii,
  // with the orbitals and envelopes of its own spin.
  const int n = full ? (s == 0 ? N : 0) : (s == 0 ? n_up : n_dn);
  const int i0 = (full || s == 0) ? 0 : n_up;
  if (n == 0) return;
  const T* gb = geo + b * E * 4;
  const T* phib = phi + b * N * Wo;
  const double bp = (double)beta[b * K + p];
  // envbar staging [Bc][spin][omega|zeta][K*nmax][M]; rows o = p*n + k.  The
  // rows of spin sr of this block are ii in [ra(sr), rb(sr)).
  const int sr0 = full ? 0 : s, sr1 = full ? 1 : s;
  auto ra = [&](int sr) { return full ? (sr == 0 ? 0 : n_up) : 0; };
  auto rb = [&](int sr) { return full ? (sr == 0 ? n_up : N) : n; };
  for (int q = lane; q < n * n; q += 32) {
    const int ii = q / n, k = q % n, o = p * n + k, i = i0 + ii;
    const bool up = i < n_up;
    const T* om = params + (up ? om_up : om_dn);
    const T* ze = params + (up ? ze_up : ze_dn);
    T ev = 0;
    for (int I = 0; I < M; ++I) ev += om[o * M + I] * exp(-ze[o * M + I] * gb[(n_ee + i * M + I) * 4]);
    env[q] = ev;
    phi0[q] = phib[(int64_t)i * Wo + o];
    LUt[q] = phi0[q] * ev;
  }
  __syncwarp();
  int sign = 0;
  double la = 0;
  bool fp64 = sizeof(T) == 8, ok = false;
  if (!fp64 && bp != 0.0) {
    if (lane < n) {
      T m = 0;
      for (int k = 0; k < n; ++k) m = max(m, (T)fabs(LUt[lane * n + k]));
      rmax[lane] = m;
    }
    __syncwarp();
    ok = warp_lu<T>(LUt, perm, n, lane, &sign, &la);
    if (ok) {
      warp_inverse<T>(LUt, perm, n, lane, Ainvt);
      T imax = 0;
      for (int q = lane; q < n * n; q += 32) imax = max(imax, (T)fabs(Ainvt[q]) * rmax[q % n]);
      fp64 = !(T(n) * warp_max(imax) <= T(10000));
    } else {
      fp64 = true;
    }
    if constexpr (sizeof(T) == 4) {
      if (!fp64) {
        // one refinement step X = X0 + X0 (I - A X0), the residual as a compensated
        // product (Dot2) into LUt, the refined inverse (error about (kappa u)^2) into Ainvt
        for (int q = lane; q < n * n; q += 32) {
          const int a = q / n, m = q % n;
          dfloat acc = {a == m ? -1.f : 0.f, 0.f};
          for (int l = 0; l < n; ++l) acc = dot2_step(acc, phi0[a * n + l] * env[a * n + l], Ainvt[l * n + m]);
          LUt[q] = -(acc.hi + acc.lo);
        }
        __syncwarp();
        for (int q = lane; q < n * n; q += 32) {  // rmax (free now) holds the refined inverse
          const int a = q / n, m = q % n;
          float c = 0.f;
          for (int l = 0; l < n; ++l) c = fmaf(Ainvt[a * n + l], LUt[l * n + m], c);
          rmax[q] = Ainvt[q] + c;
        }
        __syncwarp();
        for (int q = lane; q < n * n; q += 32) Ainvt[q] = rmax[q];
        __syncwarp();
      }
    }
  }
  if (fp64 && bp != 0.0) {
    for (int q = lane; q < n * n; q += 32) LUd[q] = (double)phi0[q] * (double)env[q];
    __syncwarp();
    ok = warp_lu<double>(LUd, perm, n, lane, &sign, &la);
    if (ok) warp_inverse<double>(LUd, perm, n, lane, Ainvd);
  }
  auto ainv = [&](int r, int c) { return fp64 ? Ainvd[r * n + c] : (double)Ainvt[r * n + c]; };
  if (!ok || bp == 0.0) {  // zero adjoint (psi = 0 or zero weight)
    for (int q = lane; q < n * n; q += 32) {
      const int ii = q / n, k = q % n;
      phibar[(b * N + i0 + ii) * (int64_t)Wo + p * n + k] = T(0);
    }
    for (int sr = sr0; sr <= sr1; ++sr) {
      T* ebo = envbar + ((b * 2 + sr) * 2 + 0) * (int64_t)K * nmax * M;
      T* ebz = envbar + ((b * 2 + sr) * 2 + 1) * (int64_t)K * nmax * M;
      for (int q = lane; q < n * M; q += 32) {
        const int k = q / M, I = q % M;
        ebo[(int64_t)(p * n + k) * M + I] = T(0);
        ebz[(int64_t)(p * n + k) * M + I] = T(0);
      }
    }
    return;
  }
  // phibar_ik = beta (A^-1)_ki env_ik
  for (int q = lane; q < n * n; q += 32) {
    const int ii = q / n, k = q % n;
    phibar[(b * N + i0 + ii) * (int64_t)Wo + p * n + k] = (T)(bp * ainv(k, ii) * (double)env[q]);
  }
  // envelope parameters of each spin present in the block: lanes over (k, I)
  for (int sr = sr0; sr <= sr1; ++sr) {
    const T* om = params + (sr == 0 ? om_up : om_dn);
    const T* ze = params + (sr == 0 ? ze_up : ze_dn);
    T* ebo = envbar + ((b * 2 + sr) * 2 + 0) * (int64_t)K * nmax * M;
    T* ebz = envbar + ((b * 2 + sr) * 2 + 1) * (int64_t)K * nmax * M;
    const int iia = ra(sr), iib = rb(sr);
    for (int q = lane; q < n * M; q += 32) {
      const int k = q / M, I = q % M, o = p * n + k;
      const T w = om[o * M + I], z = ze[o * M + I];
      T ob = 0, zb = 0;
      for (int ii = iia; ii < iib; ++ii) {
        const int i = i0 + ii;
        const T d = gb[(n_ee + i * M + I) * 4];
        const T e = exp(-z * d);
        const T envb = (T)(bp * ainv(k, ii)) * phi0[ii * n + k];
        ob += envb * e;
        zb -= envb * w * d * e;
      }
      ebo[(int64_t)o * M + I] = ob;
      ebz[(int64_t)o * M + I] = zb;
    }
  }
}

// ---------------------------------------------------------------------------
// Y[r][n] (+)= sum_k X[r][k] W[k][n]   (W row-major [K][n_out]), any sizes.
// ---------------------------------------------------------------------------
constexpr int NB = 64, NK = 16;
template <class T>
__global__ void __launch_bounds__(256)
    gemm_nn_kernel(const T* __restrict__ X, RowMap mx, const T* __restrict__ W, T* __restrict__ Y, RowMap my,
                   int64_t rows, int n_out, int K, int accumulate) {
  __shared__ T Xs[NK][NB + 1];
  __shared__ T Ws[NK][NB + 1];
  __shared__ int64_t xoff[NB], yoff[NB];  // row offsets of this tile (one division per row)
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t r0 = (int64_t)blockIdx.x * NB;
  const int n0 = blockIdx.y * NB;
  if (threadIdx.x < NB) {
    const int64_t r = r0 + threadIdx.x;
    xoff[threadIdx.x] = r < rows ? (r / mx.rows_per_seg) * mx.seg_stride + (r % mx.rows_per_seg) * mx.ld : -1;
    yoff[threadIdx.x] = r < rows ? (r / my.rows_per_seg) * my.seg_stride + (r % my.rows_per_seg) * my.ld : -1;
  }
  __syncthreads();
  T acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += NK) {
    for (int e = threadIdx.x; e < NB * NK; e += 256) {
      const int rr = e / NK, kk = e % NK;
      const int k = k0 + kk;
      const int64_t xo = xoff[rr];
      Xs[kk][rr] = (xo >= 0 && k < K) ? X[xo + k] : T(0);
      const int kk2 = e / NB, nn2 = e % NB;
      const int k2 = k0 + kk2, n2 = n0 + nn2;
      Ws[kk2][nn2] = (k2 < K && n2 < n_out) ? W[(int64_t)k2 * n_out + n2] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < NK; ++kk) {
      T a[4], w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Xs[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = Ws[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * w[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t yo = yoff[ty + 16 * i];
    if (yo < 0) continue;
    T* y = Y + yo;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n < n_out) y[n] = accumulate ? y[n] + acc[i][j] : acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------
// Parameter reduction over rows:
//   S_b[o][a] = sum_{r < rpw} X[b,r][o] * (Y ? Y[b,r][a] : 1)
// per walker (mode 1): G[b][off + o*ld + a] = S_b
// weighted   (mode 0): part[split][o][a] = sum over the split's walkers,
//                      then reduce_splits adds sum_split part to G[off + ...].
// Rows of walker b: row index b*rpw + r through the row maps.
// ---------------------------------------------------------------------------
constexpr int RT = 32;  // output tile (o, a)
template <class T>
__global__ void __launch_bounds__(256)
    param_reduce_kernel(const T* __restrict__ X, RowMap mx, const T* __restrict__ Y, RowMap my, int rpw, int64_t nw,
                        int n_o, int n_a, T* __restrict__ G, int64_t P, int64_t off, int ld, int mode,
                        int64_t walkers_per_split, T* __restrict__ part) {
  __shared__ T Xs[8][RT + 1];
  __shared__ T Ys[8][RT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int o0 = blockIdx.x * RT, a0 = blockIdx.y * RT;
  int64_t wb0, wb1;
  if (mode == 1) {
    wb0 = blockIdx.z;
    wb1 = wb0 + 1;
  } else {
    wb0 = (int64_t)blockIdx.z * walkers_per_split;
    wb1 = min(nw, wb0 + walkers_per_split);
  }
  const int64_t r_begin = wb0 * rpw, r_end = wb1 * rpw;
  T acc[2][2] = {};
  for (int64_t rr0 = r_begin; rr0 < r_end; rr0 += 8) {
    for (int e = threadIdx.x; e < 8 * RT; e += 256) {
      const int k = e / RT, c = e % RT;
      const int64_t r = rr0 + k;
      const bool ok = r < r_end;
      const int o = o0 + c, a = a0 + c;
      Xs[k][c] = (ok && o < n_o) ? X[(r / mx.rows_per_seg) * mx.seg_stride + (r % mx.rows_per_seg) * mx.ld + o] : T(0);
      Ys[k][c] = (ok && a < n_a) ? (Y ? Y[(r / my.rows_per_seg) * my.seg_stride + (r % my.rows_per_seg) * my.ld + a]
                                      : T(1))
                                 : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const T x0 = Xs[k][ty], x1 = Xs[k][ty + 16];
      const T y0 = Ys[k][tx], y1 = Ys[k][tx + 16];
      acc[0][0] += x0 * y0;
      acc[0][1] += x0 * y1;
      acc[1][0] += x1 * y0;
      acc[1][1] += x1 * y1;
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int o = o0 + ty + 16 * i, a = a0 + tx + 16 * j;
      if (o >= n_o || a >= n_a) continue;
      if (mode == 1)
        G[wb0 * P + off + (int64_t)o * ld + a] = acc[i][j];
      else
        part[((int64_t)blockIdx.z * n_o + o) * n_a + a] = acc[i][j];
    }
}

// Large parameter blocks: Out[o][a] = sum_r X[r][o] Y[r][a] as a tiled GEMM
// whose reduction index is the row index.  Rows are the slow index of both
// operands, so BK consecutive rows of X and Y are copied into shared memory
// as they are ([k][o], [k][a]); each thread accumulates a TM x TN register
// block (split halves, conflict-free reads).  blockIdx.z selects a walker
// (per-walker mode, output G + b*P) or a split of the walker range
// (summed mode, output part[split]).
template <class T>
struct VecT;
template <>
struct VecT<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct VecT<double> {
  using type = double2;
  static constexpr int n = 2;
};

template <class T, int BM, int BN, int BK, bool VA>
__global__ void __launch_bounds__(256)
    gemm_tn_kernel(const T* __restrict__ X, RowMap mx, const T* __restrict__ Y, RowMap my, int rpw, int64_t nw,
                   int n_o, int n_a, T* __restrict__ G, int64_t P, int64_t off, int ld, int mode,
                   int64_t walkers_per_split, T* __restrict__ part) {
  using V = typename VecT<T>::type;
  constexpr int VEC = VecT<T>::n;
  constexpr int TM = 2 * VEC, TN = 2 * VEC;
  static_assert((BM / TM) * (BN / TN) == 256, "tile/thread mismatch");
  __shared__ __align__(16) T Xs[BK][BM];
  __shared__ __align__(16) T Ys[BK][BN];
  __shared__ int64_t xoff[BK], yoff[BK];  // offsets of the BK rows of this step
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int o0 = blockIdx.x * BM, a0 = blockIdx.y * BN;
  int64_t wb0, wb1;
  if (mode == 1) {
    wb0 = blockIdx.z;
    wb1 = wb0 + 1;
  } else {
    wb0 = (int64_t)blockIdx.z * walkers_per_split;
    wb1 = min(nw, wb0 + walkers_per_split);
  }
  const int64_t r_begin = wb0 * rpw, r_end = wb1 * rpw;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  constexpr int XV = BM / VEC, YV = BN / VEC;  // vectors per row of a tile
  for (int64_t rr0 = r_begin; rr0 < r_end; rr0 += BK) {
    if (tid < BK) {
      const int64_t r = rr0 + tid;
      xoff[tid] = r < r_end ? (r / mx.rows_per_seg) * mx.seg_stride + (r % mx.rows_per_seg) * mx.ld : -1;
      yoff[tid] = r < r_end ? (r / my.rows_per_seg) * my.seg_stride + (r % my.rows_per_seg) * my.ld : -1;
    }
    __syncthreads();
    for (int e = tid; e < BK * XV; e += 256) {
      const int k = e / XV, cv = e % XV;
      const int o = o0 + cv * VEC;
      V v{};
      if (xoff[k] >= 0) {
        const T* src = X + xoff[k] + o;
        if (VA && o + VEC <= n_o) {
          v = *reinterpret_cast<const V*>(src);
        } else {
          T* t = reinterpret_cast<T*>(&v);
          for (int q = 0; q < VEC; ++q) t[q] = o + q < n_o ? src[q] : T(0);
        }
      }
      *reinterpret_cast<V*>(&Xs[k][cv * VEC]) = v;
    }
    for (int e = tid; e < BK * YV; e += 256) {
      const int k = e / YV, cv = e % YV;
      const int a = a0 + cv * VEC;
      V v{};
      if (yoff[k] >= 0) {
        const T* src = Y + yoff[k] + a;
        if (VA && a + VEC <= n_a) {
          v = *reinterpret_cast<const V*>(src);
        } else {
          T* t = reinterpret_cast<T*>(&v);
          for (int q = 0; q < VEC; ++q) t[q] = a + q < n_a ? src[q] : T(0);
        }
      }
      *reinterpret_cast<V*>(&Ys[k][cv * VEC]) = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T x[TM], y[TN];
      *reinterpret_cast<V*>(&x[0]) = *reinterpret_cast<const V*>(&Xs[kk][ty * VEC]);
      *reinterpret_cast<V*>(&x[VEC]) = *reinterpret_cast<const V*>(&Xs[kk][BM / 2 + ty * VEC]);
      *reinterpret_cast<V*>(&y[0]) = *reinterpret_cast<const V*>(&Ys[kk][tx * VEC]);
      *reinterpret_cast<V*>(&y[VEC]) = *reinterpret_cast<const V*>(&Ys[kk][BN / 2 + tx * VEC]);
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(x[i], y[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int o = o0 + ((i < VEC) ? ty * VEC + i : BM / 2 + ty * VEC + (i - VEC));
    if (o >= n_o) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int a = a0 + ((j < VEC) ? tx * VEC + j : BN / 2 + tx * VEC + (j - VEC));
      if (a >= n_a) continue;
      if (mode == 1)
        G[wb0 * P + off + (int64_t)o * ld + a] = acc[i][j];
      else
        part[((int64_t)blockIdx.z * n_o + o) * n_a + a] = acc[i][j];
    }
  }
}

// Column sums S[o] = sum_r X[r][o] (bias-type gradients).  A CTA covers 32
// consecutive columns (one per lane, coalesced rows) with 8 warps that take
// every 8th row of the walker range; the 8 partial sums are added in a fixed
// order in shared memory.  blockIdx.y: walker (per-walker mode) or split.
constexpr int kColRows = 8;
constexpr int kColsumCounters = kColsumReduceCounters;  // column blocks of one column sum (n_o <= 2048)
template <class T>
__global__ void __launch_bounds__(32 * kColRows)
    colsum_kernel(const T* __restrict__ X, RowMap mx, int rpw, int64_t nw, int n_o, T* __restrict__ G, int64_t P,
                  int64_t off, int ld, int mode, int64_t walkers_per_split, T* __restrict__ part,
                  unsigned int* __restrict__ done) {
  __shared__ T red[kColRows][32];
  const int lane = threadIdx.x % 32, rl = threadIdx.x / 32;
  const int o = blockIdx.x * 32 + lane;
  int64_t wb0, wb1;
  if (mode == 1) {
    wb0 = blockIdx.y;
    wb1 = wb0 + 1;
  } else {
    wb0 = (int64_t)blockIdx.y * walkers_per_split;
    wb1 = min(nw, wb0 + walkers_per_split);
  }
  T acc = 0;
  const int64_t r_begin = wb0 * rpw + rl, r_end = wb1 * rpw;
  if (o < n_o && r_begin < r_end) {
    const T* xo = X + o;
    if (r_end <= (int64_t)UINT32_MAX && mx.rows_per_seg <= (int64_t)UINT32_MAX) {
      // kColU rows per iteration, each addressed on its own (32-bit division) and summed into
      // its own accumulator, so that kColU loads are in flight; the accumulators are added in
      // a fixed order
      constexpr int kColU = 8;
      const uint32_t rps = (uint32_t)mx.rows_per_seg;
      T a[kColU];
#pragma unroll
      for (int u = 0; u < kColU; ++u) a[u] = 0;
      for (int64_t r0 = r_begin; r0 < r_end; r0 += (int64_t)kColU * kColRows) {
        T v[kColU];
#pragma unroll
        for (int u = 0; u < kColU; ++u) {
          const int64_t r = r0 + (int64_t)u * kColRows;
          const uint32_t seg = (uint32_t)r / rps, in = (uint32_t)r - seg * rps;
          v[u] = r < r_end ? xo[(int64_t)seg * mx.seg_stride + (int64_t)in * mx.ld] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kColU; ++u) a[u] += v[u];
      }
#pragma unroll
      for (int u = 0; u < kColU; ++u) acc += a[u];
    } else {
      int64_t seg = r_begin / mx.rows_per_seg, in = r_begin % mx.rows_per_seg;  // one division, then increments
      for (int64_t r = r_begin; r < r_end; r += kColRows) {
        acc += xo[seg * mx.seg_stride + in * mx.ld];
        in += kColRows;
        while (in >= mx.rows_per_seg) {
          in -= mx.rows_per_seg;
          ++seg;
        }
      }
    }
  }
  red[rl][lane] = acc;
  __syncthreads();
  if (rl == 0 && o < n_o) {
    T sum = 0;
#pragma unroll
    for (int k = 0; k < kColRows; ++k) sum += red[k][lane];
    if (mode == 1)
      G[wb0 * P + off + (int64_t)o * ld] = sum;
    else
      part[(int64_t)blockIdx.y * n_o + o] = sum;
  }
  if (mode == 1 || done == nullptr) return;
  // The last split CTA of this column block adds the splits in order (deterministic).
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&done[blockIdx.x], 1u) == gridDim.y - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (rl == 0 && o < n_o) {
    T sum = 0;
    for (unsigned sp = 0; sp < gridDim.y; ++sp) sum += __ldcg(part + (int64_t)sp * n_o + o);
    G[off + (int64_t)o * ld] += sum;
  }
  if (threadIdx.x == 0) done[blockIdx.x] = 0;  // ready for the next use of this counter
}

template <class T>
__global__ void reduce_splits_kernel(const T* __restrict__ part, int splits, int n_o, int n_a, T* __restrict__ G,
                                     int64_t off, int ld) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n_o * n_a) return;
  T acc = 0;
  for (int s = 0; s < splits; ++s) acc += part[(int64_t)s * n_o * n_a + e];
  const int o = (int)(e / n_a), a = (int)(e % n_a);
  G[off + (int64_t)o * ld + a] += acc;
}

// out[r][a] = g[r][a] * (1 - t^2), t = tanh(u[r][a]) (is_tanh_of_u) or t = u.
template <class T>
__global__ void tanh_bwd_kernel(const T* __restrict__ g, const T* __restrict__ u, int64_t n, int is_pre,
                                T* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const T t = is_pre ? tanh(u[e]) : u[e];
  out[e] = g[e] * (T(1) - t * t);
}

// fbar[b][i][a] += sbar[b][a] for every electron i (the Jastrow input is sum_i f_i).
template <class T>
__global__ void add_rows_kernel(T* __restrict__ fbar, const T* __restrict__ sbar, int64_t Bc, int N, int D) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Bc * N * D) return;
  const int64_t b = e / (N * D);
  fbar[e] += sbar[b * D + e % D];
}

// ---------------------------------------------------------------------------
// Message backward, Eq. (17).  One CTA per (walker, chunk of DC features);
// thread (feature lane, sender j).  With m_i^t = nu_t(i) sum_j w_ij z_j:
//   zbar_j   = sum_{i != j} nu_{t(i,j)}(i) mbar_i^{t(i,j)} w_ij
//   wbar_ij  = nu(i) mbar_i^t z_j + nu(j) mbar_j^t z_i       (pair p = (i, j))
//   wbar_iI  = mbar_i^nuc Y_I / M,   Ybar_I = sum_i mbar_i^nuc w_iI / M
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256)
    msg_bwd_kernel(const T* __restrict__ mbar, const T* __restrict__ Z, const T* __restrict__ z0,
                   const T* __restrict__ ew, const T* __restrict__ Y, const int* __restrict__ pair_ij,
                   const int* __restrict__ pair_of, int N, int n_up,
                   int M, int D, int E, int n_ee, int z_const, T* __restrict__ zbar, T* __restrict__ wbar,
                   T* __restrict__ ybar) {
  extern __shared__ __align__(16) unsigned char msg_bwd_raw[];
  const int64_t b = blockIdx.x;
  const int L = 32;
  T* Ms = reinterpret_cast<T*>(msg_bwd_raw);  // [N][2][L] normalised same / opposite message adjoints
  T* Zs = Ms + N * 2 * L;                      // [N][L] z_j
  int* Po = reinterpret_cast<int*>(Zs + N * L);  // [N][N] pair index
  int* Pij = Po + N * N;                          // [n_ee][2] electrons of a pair
  const int dl = threadIdx.x % 32, d = blockIdx.y * 32 + dl;
  const int grp = threadIdx.x / 32, ngrp = blockDim.x / 32;
  const int n_dn = N - n_up;
  const T* mb = mbar + b * N * 3 * D;
  const T* ewb = ew + b * E * D;
  for (int k = threadIdx.x; k < N * N; k += blockDim.x) Po[k] = pair_of[k];
  for (int k = threadIdx.x; k < 2 * n_ee; k += blockDim.x) Pij[k] = pair_ij[k];
  for (int i = grp; i < N; i += ngrp) {
    const int ns = i < n_up ? n_up : n_dn, no = N - ns;
    const T nus = T(1) / T(ns - 1 > 1 ? ns - 1 : 1), nuo = T(1) / T(no > 1 ? no : 1);
    Ms[(i * 2 + 0) * L + dl] = d < D ? mb[(int64_t)i * 3 * D + d] * nus : T(0);
    Ms[(i * 2 + 1) * L + dl] = d < D ? mb[(int64_t)i * 3 * D + D + d] * nuo : T(0);
    Zs[i * L + dl] = d >= D ? T(0) : (z_const ? z0[(i < n_up ? 0 : 1) * D + d] : Z[(b * N + i) * D + d]);
  }
  __syncthreads();
  if (d >= D) return;
  auto m_in = [&](int i, int j) {  // mbar_i^t for the edge (i, j), normalised
    return Ms[(i * 2 + ((i < n_up) == (j < n_up) ? 0 : 1)) * L + dl];
  };
  auto zv = [&](int j) { return Zs[j * L + dl]; };
  // zbar_j (independent loads, several in flight)
  for (int j = grp; j < N; j += ngrp) {
    T acc = 0;
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
      if (i == j) continue;
      acc += m_in(i, j) * ewb[(int64_t)Po[i * N + j] * D + d];
    }
    zbar[(b * N + j) * D + d] = acc;
  }
  // wbar for e-e pairs
#pragma unroll 4
  for (int e = grp; e < n_ee; e += ngrp) {
    const int i = Pij[2 * e], j = Pij[2 * e + 1];
    wbar[(b * E + e) * D + d] = m_in(i, j) * zv(j) + m_in(j, i) * zv(i);
  }
  // electron-nucleus edges and Ybar
  const T nuM = T(1) / T(M);
  for (int e = n_ee + grp; e < E; e += ngrp) {
    const int i = (e - n_ee) / M, I = (e - n_ee) % M;
    wbar[(b * E + e) * D + d] = mb[(int64_t)i * 3 * D + 2 * D + d] * nuM * Y[(int64_t)I * D + d];
  }
  for (int I = grp; I < M; I += ngrp) {
    T acc = 0;
    for (int i = 0; i < N; ++i) acc += mb[(int64_t)i * 3 * D + 2 * D + d] * ewb[(int64_t)(n_ee + i * M + I) * D + d];
    ybar[(b * M + I) * D + d] = acc * nuM;
  }
}

// F0[b][i][a] = E_spin[sigma_i][a]: the layer-0 embeddings of Eq. (13).
template <class T>
__global__ void fill_spin_rows_kernel(T* __restrict__ F0, const T* __restrict__ E_spin, int64_t Bc, int N, int n_up,
                                      int D) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Bc * N * D) return;
  const int i = (int)((e / D) % N);
  F0[e] = E_spin[(i < n_up ? 0 : 1) * D + e % D];
}

// ---------------------------------------------------------------------------
// Reverse of one layer's edge-embedding update f^l = f + tanh(U f + c) (value
// rows): with th = tanh(U f + c) recomputed from the saved input f = f^{l-1},
//   abar = ebar (1 - th^2)        (adjoint of U f + c: U-bar = abar f^T, c-bar = abar)
//   ebar <- ebar + U^T abar       (adjoint of f^{l-1}: the identity path plus the map)
// ebar is updated in place; one thread per (row, feature), rows staged in
// shared memory.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256)
    edge_update_bwd_kernel(const T* __restrict__ fprev, T* __restrict__ ebar, T* __restrict__ abar,
                           const T* __restrict__ params, int64_t Bc, int E, int n_par, int n_ee, int Q, int64_t U0,
                           int64_t U1, int64_t U2, int64_t c0, int64_t c1, int64_t c2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Us = reinterpret_cast<T*>(smem_raw);  // [3][Q][Q]
  T* cs = Us + 3 * Q * Q;                  // [3][Q]
  const int rpi = blockDim.x / Q;
  T* fs = cs + 3 * Q;   // [rpi][Q]
  T* es = fs + rpi * Q;  // [rpi][Q]
  T* as = es + rpi * Q;  // [rpi][Q]
  const int64_t Uo[3] = {U0, U1, U2}, co[3] = {c0, c1, c2};
  for (int t = 0; t < 3; ++t) {
    for (int k = threadIdx.x; k < Q * Q; k += blockDim.x) Us[t * Q * Q + k] = params[Uo[t] + k];
    for (int k = threadIdx.x; k < Q; k += blockDim.x) cs[t * Q + k] = params[co[t] + k];
  }
  const int rr = threadIdx.x / Q, q = threadIdx.x % Q;
  const int64_t nrows = Bc * E;
  for (int64_t be0 = (int64_t)blockIdx.x * rpi; be0 < nrows; be0 += (int64_t)gridDim.x * rpi) {
    const int nb = (int)min((int64_t)rpi, nrows - be0);
    __syncthreads();
    for (int k = threadIdx.x; k < nb * Q; k += blockDim.x) {
      fs[k] = fprev[be0 * Q + k];
      es[k] = ebar[be0 * Q + k];
    }
    __syncthreads();
    const bool live = rr < nb;
    const int64_t be = be0 + rr;
    const int e = (int)(be % E);
    const int t = e < n_par ? 0 : (e < n_ee ? 1 : 2);
    if (live) {
      const T* f = fs + rr * Q;
      const T* u = Us + (t * Q + q) * Q;
      T v = cs[t * Q + q];
      for (int k = 0; k < Q; ++k) v += u[k] * f[k];
      const T th = tanh(v);
      const T ab = es[rr * Q + q] * (T(1) - th * th);
      as[rr * Q + q] = ab;
      abar[be * Q + q] = ab;
    }
    __syncthreads();
    if (live) {
      T acc = es[rr * Q + q];
      for (int j = 0; j < Q; ++j) acc += Us[(t * Q + j) * Q + q] * as[rr * Q + j];
      ebar[be * Q + q] = acc;
    }
  }
}

}  // namespace

template <class T>
cudaError_t launch_edge_update_bwd(const dq_handle_s& h, int64_t Bc, int l, const T* params, const T* fprev, T* ebar,
                                   T* abar, cudaStream_t s) {
  const int Q = h.Q, rpi = 256 / Q;
  const auto& y = h.off.layer[l];
  const int64_t rows = Bc * h.edges.n_all, nblk = (rows + rpi - 1) / rpi;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = ((size_t)3 * Q * Q + 3 * Q + (size_t)3 * rpi * Q) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(edge_update_bwd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nblk, (int64_t)std::max(sms, 1) * 8));
  edge_update_bwd_kernel<T><<<grid, 256, smem, s>>>(fprev, ebar, abar, params, Bc, h.edges.n_all, h.edges.n_par,
                                                    h.edges.n_ee, Q, y.U[0], y.U[1], y.U[2], y.c[0], y.c[1],
                                                    y.c[2]);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_fill_spin_rows(T* F0, const T* E_spin, int64_t Bc, int N, int n_up, int D, cudaStream_t s) {
  fill_spin_rows_kernel<T><<<nblocks(Bc * N * D, 256), 256, 0, s>>>(F0, E_spin, Bc, N, n_up, D);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <class T>
cudaError_t launch_bwd_combine(const dq_handle_s& h, int64_t Bc, const double* det, const T* jh, const T* params,
                               const T* weights, T* beta, T* cbar, T* jhbar, T* gt, cudaStream_t s) {
  bwd_combine_kernel<T><<<nblocks(Bc * 32, 128), 128, 0, s>>>(det, jh, params, weights, Bc, h.N, h.K, h.D, h.off.c,
                                                             h.off.w_J2, h.use_jastrow, beta, cbar, jhbar, gt);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_bwd_det(const dq_handle_s& h, int64_t Bc, const T* phi, const T* geo, const T* params, const T* beta,
                           T* phibar, T* envbar, cudaStream_t s) {
  const int nmax = h.det_n();
  const int nn = nmax * nmax;
  const size_t per_warp = ((size_t)nn * (2 * sizeof(double) + 5 * sizeof(T)) + 32 * sizeof(int) + 15) / 16 * 16;
  const int warps = 4;
  const size_t smem = per_warp * warps;
  auto kern = bwd_det_kernel<T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nblocks(Bc * 2 * h.K, warps), warps * 32, smem, s>>>(
      phi, geo, params, beta, Bc, h.N, h.n_up, h.M, h.K, h.K * nmax, h.edges.n_all, h.edges.n_ee, h.off.omega[0],
      h.off.omega[1], h.off.zeta[0], h.off.zeta[1], phibar, envbar, h.full_det);
  return cudaGetLastError();
}

template <class T>
cudaError_t gemm_nn(const T* X, RowMap mx, const T* W, T* Y, RowMap my, int64_t rows, int n_out, int K,
                    bool accumulate, cudaStream_t s) {
  if (rows <= 0 || n_out <= 0 || K <= 0) return cudaSuccess;
  dim3 grid(nblocks(rows, NB), nblocks(n_out, NB));
  gemm_nn_kernel<T><<<grid, 256, 0, s>>>(X, mx, W, Y, my, rows, n_out, K, accumulate ? 1 : 0);
  return cudaGetLastError();
}

template <class T>
cudaError_t param_reduce_tiled(const T* X, RowMap mx, const T* Y, RowMap my, int rpw, int64_t nw, int n_o, int n_a,
                               T* G, int64_t P, int64_t off, int ld, int mode, T* part, int64_t part_elems,
                               cudaStream_t s) {
  constexpr int BM = sizeof(T) == 4 ? 128 : 64, BN = BM, BK = 8;
  constexpr int VEC = VecT<T>::n;
  const bool va = (uintptr_t)X % 16 == 0 && (uintptr_t)Y % 16 == 0 && mx.ld % VEC == 0 && my.ld % VEC == 0 &&
                  mx.seg_stride % VEC == 0 && my.seg_stride % VEC == 0;
  const unsigned gx = nblocks(n_o, BM), gy = nblocks(n_a, BN);
  auto launch = [&](dim3 grid, const T* Xo, const T* Yo, int64_t nws, T* Go, int md, int64_t wps, T* pt) {
    if (va)
      gemm_tn_kernel<T, BM, BN, BK, true><<<grid, 256, 0, s>>>(Xo, mx, Yo, my, rpw, nws, n_o, n_a, Go, P, off, ld, md,
                                                                wps, pt);
    else
      gemm_tn_kernel<T, BM, BN, BK, false><<<grid, 256, 0, s>>>(Xo, mx, Yo, my, rpw, nws, n_o, n_a, Go, P, off, ld, md,
                                                                 wps, pt);
  };
  if (mode == 1) {
    for (int64_t w0 = 0; w0 < nw; w0 += 65535) {
      const int64_t nws = nw - w0 < 65535 ? nw - w0 : 65535;
      const int64_t r_off = w0 * rpw;
      const T* Xo = X + (r_off / mx.rows_per_seg) * mx.seg_stride + (r_off % mx.rows_per_seg) * mx.ld;
      const T* Yo = Y + (r_off / my.rows_per_seg) * my.seg_stride + (r_off % my.rows_per_seg) * my.ld;
      launch(dim3(gx, gy, (unsigned)nws), Xo, Yo, nws, G + w0 * P, 1, 1, nullptr);
    }
    return cudaGetLastError();
  }
  // summed over walkers: about 2 CTAs per SM in total, deterministic second pass
  const int64_t per = (int64_t)n_o * n_a;
  int64_t splits = (304 + gx * gy - 1) / (gx * gy);
  if (splits > nw) splits = nw;
  if (splits * per > part_elems) splits = part_elems / per;
  if (splits < 1) return cudaErrorInvalidValue;
  const int64_t wps = (nw + splits - 1) / splits;
  splits = (nw + wps - 1) / wps;
  launch(dim3(gx, gy, (unsigned)splits), X, Y, nw, G, 0, wps, part);
  reduce_splits_kernel<T><<<nblocks(per, 256), 256, 0, s>>>(part, (int)splits, n_o, n_a, G, off, ld);
  return cudaGetLastError();
}

// Row maps as (rows per walker, row pitch, walker stride), or false if the rows of a
// walker are not equally spaced.
inline bool walker_rows(RowMap m, int rpw, int64_t* pitch, int64_t* wstride) {
  if (m.rows_per_seg == 1) {
    *pitch = m.seg_stride;
    *wstride = (int64_t)rpw * m.seg_stride;
    return true;
  }
  if (m.rows_per_seg == rpw) {
    *pitch = m.ld;
    *wstride = m.seg_stride;
    return true;
  }
  return false;
}

template <class T>
cudaError_t param_reduce(const T* X, RowMap mx, const T* Y, RowMap my, int rpw, int64_t nw, int n_o, int n_a, T* G,
                         int64_t P, int64_t off, int ld, int mode, T* part, int64_t part_elems, cudaStream_t s,
                         unsigned int* tc_status, unsigned int* done, int64_t boff, bool* bias_done) {
  if (bias_done) *bias_done = false;
  if (nw <= 0 || n_o <= 0 || n_a <= 0) return cudaSuccess;
  if (rpw <= 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    int64_t xp, xs, yp, ys, splits = 0;
    if (tc_status != nullptr && mode == 0 && Y != nullptr && n_o >= 64 && n_a >= 16 &&
        walker_rows(mx, rpw, &xp, &xs) && walker_rows(my, rpw, &yp, &ys)) {
      float* colpart = nullptr;
      const cudaError_t e = gemm_tn_tf32x3(X, xp, xs, Y, yp, ys, rpw, nw, n_o, n_a, part, part_elems, &splits,
                                           tc_status, s, boff >= 0 && bias_done ? &colpart : nullptr);
      if (e == cudaSuccess && splits > 0) {
        const int64_t per = (int64_t)n_o * n_a;
        reduce_splits_kernel<T><<<nblocks(per, 256), 256, 0, s>>>(part, (int)splits, n_o, n_a, G, off, ld);
        if (colpart != nullptr) {
          reduce_splits_kernel<T><<<nblocks(n_o, 256), 256, 0, s>>>(colpart, (int)splits, n_o, 1, G, boff, 1);
          *bias_done = true;
        }
        return cudaGetLastError();
      }
      if (e != cudaErrorInvalidValue) return e;  // unsupported layout: the CUDA-core path below
    }
  }
  if (Y != nullptr && n_o >= 16 && n_a >= 16)
    return param_reduce_tiled<T>(X, mx, Y, my, rpw, nw, n_o, n_a, G, P, off, ld, mode, part, part_elems, s);
  if (Y == nullptr && n_a == 1) {
    const unsigned gx = nblocks(n_o, 32);
    if (mode == 1) {
      for (int64_t w0 = 0; w0 < nw; w0 += 65535) {
        const int64_t nws = nw - w0 < 65535 ? nw - w0 : 65535;
        const int64_t r_off = w0 * rpw;
        const T* Xo = X + (r_off / mx.rows_per_seg) * mx.seg_stride + (r_off % mx.rows_per_seg) * mx.ld;
        colsum_kernel<T><<<dim3(gx, (unsigned)nws), 32 * kColRows, 0, s>>>(Xo, mx, rpw, nws, n_o, G + w0 * P, P, off,
                                                                          ld, 1, 1, nullptr, nullptr);
      }
      return cudaGetLastError();
    }
    int64_t splits = (4 * 152 + gx - 1) / gx;  // about four CTAs per SM
    if (splits > nw) splits = nw;
    if (splits * n_o > part_elems) splits = part_elems / n_o;
    if (splits < 1) return cudaErrorInvalidValue;
    if (splits > 65535) splits = 65535;
    const int64_t wps = (nw + splits - 1) / splits;
    splits = (nw + wps - 1) / wps;
    if (done != nullptr && gx <= kColsumCounters) {
      colsum_kernel<T><<<dim3(gx, (unsigned)splits), 32 * kColRows, 0, s>>>(X, mx, rpw, nw, n_o, G, P, off, ld, 0,
                                                                            wps, part, done);
    } else {
      colsum_kernel<T><<<dim3(gx, (unsigned)splits), 32 * kColRows, 0, s>>>(X, mx, rpw, nw, n_o, G, P, off, ld, 0,
                                                                            wps, part, nullptr);
      reduce_splits_kernel<T><<<nblocks(n_o, 256), 256, 0, s>>>(part, (int)splits, n_o, 1, G, off, ld);
    }
    return cudaGetLastError();
  }
  const unsigned gx = nblocks(n_o, RT), gy = nblocks(n_a, RT);
  if (mode == 1) {
    // grid.z is limited to 65535: loop over walker slices
    for (int64_t w0 = 0; w0 < nw; w0 += 65535) {
      const int64_t nws = nw - w0 < 65535 ? nw - w0 : 65535;
      dim3 grid(gx, gy, (unsigned)nws);
      // offset the row maps by whole walkers: rows of walker w0 start at w0*rpw
      const int64_t r_off = w0 * rpw;
      const T* Xo = X + (r_off / mx.rows_per_seg) * mx.seg_stride + (r_off % mx.rows_per_seg) * mx.ld;
      const T* Yo = Y ? Y + (r_off / my.rows_per_seg) * my.seg_stride + (r_off % my.rows_per_seg) * my.ld : nullptr;
      param_reduce_kernel<T><<<grid, 256, 0, s>>>(Xo, mx, Yo, my, rpw, nws, n_o, n_a, G + w0 * P, P, off, ld, 1, 1,
                                                  nullptr);
    }
    return cudaGetLastError();
  }
  // weighted: choose the split count so that the partial sums fit the scratch
  int64_t splits = (nw + 63) / 64;
  const int64_t per = (int64_t)n_o * n_a;
  if (splits * per > part_elems) splits = part_elems / per;
  if (splits < 1) return cudaErrorInvalidValue;
  if (splits > 65535) splits = 65535;
  const int64_t wps = (nw + splits - 1) / splits;
  splits = (nw + wps - 1) / wps;
  dim3 grid(gx, gy, (unsigned)splits);
  param_reduce_kernel<T><<<grid, 256, 0, s>>>(X, mx, Y, my, rpw, nw, n_o, n_a, G, P, off, ld, 0, wps, part);
  reduce_splits_kernel<T><<<nblocks(per, 256), 256, 0, s>>>(part, (int)splits, n_o, n_a, G, off, ld);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_tanh_bwd(const T* g, const T* u, int64_t n, bool is_pre, T* out, cudaStream_t s) {
  tanh_bwd_kernel<T><<<nblocks(n, 256), 256, 0, s>>>(g, u, n, is_pre ? 1 : 0, out);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_add_rows(T* fbar, const T* sbar, int64_t Bc, int N, int D, cudaStream_t s) {
  add_rows_kernel<T><<<nblocks(Bc * N * D, 256), 256, 0, s>>>(fbar, sbar, Bc, N, D);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_msg_bwd(const dq_handle_s& h, int64_t Bc, const T* mbar, const T* Z, const T* z0, const T* ew,
                           const T* Y, bool z_const, T* zbar, T* wbar, T* ybar, cudaStream_t s) {
  dim3 grid((unsigned)Bc, nblocks(h.D, 32));
  const size_t smem = (size_t)h.N * 3 * 32 * sizeof(T) + (size_t)(h.N * h.N + 2 * h.edges.n_ee) * sizeof(int);
  msg_bwd_kernel<T><<<grid, 256, smem, s>>>(mbar, Z, z0, ew, Y, h.d_pair_ij, h.d_pair_of, h.N, h.n_up, h.M, h.D, h.edges.n_all,
                                          h.edges.n_ee, z_const ? 1 : 0, zbar, wbar, ybar);
  return cudaGetLastError();
}

#define DQ_BWD_INST(T)                                                                                             \
  template cudaError_t launch_bwd_combine<T>(const dq_handle_s&, int64_t, const double*, const T*, const T*,       \
                                             const T*, T*, T*, T*, T*, cudaStream_t);                             \
  template cudaError_t launch_bwd_det<T>(const dq_handle_s&, int64_t, const T*, const T*, const T*, const T*, T*, \
                                         T*, cudaStream_t);                                                       \
  template cudaError_t gemm_nn<T>(const T*, RowMap, const T*, T*, RowMap, int64_t, int, int, bool, cudaStream_t); \
  template cudaError_t param_reduce<T>(const T*, RowMap, const T*, RowMap, int, int64_t, int, int, T*, int64_t,   \
                                       int64_t, int, int, T*, int64_t, cudaStream_t, unsigned int*,              \
                                       unsigned int*, int64_t, bool*);                                            \
  template cudaError_t launch_tanh_bwd<T>(const T*, const T*, int64_t, bool, T*, cudaStream_t);                   \
  template cudaError_t launch_add_rows<T>(T*, const T*, int64_t, int, int, cudaStream_t);                         \
  template cudaError_t launch_edge_update_bwd<T>(const dq_handle_s&, int64_t, int, const T*, const T*, T*, T*,    \
                                                 cudaStream_t);                                                   \
  template cudaError_t launch_fill_spin_rows<T>(T*, const T*, int64_t, int, int, int, cudaStream_t);              \
  template cudaError_t launch_msg_bwd<T>(const dq_handle_s&, int64_t, const T*, const T*, const T*, const T*,     \
                                         const T*, bool, T*, T*, T*, cudaStream_t);
DQ_BWD_INST(float)
DQ_BWD_INST(double)

}  // namespace dq
