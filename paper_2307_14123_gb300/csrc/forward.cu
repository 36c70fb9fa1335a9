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
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include <type_traits>

#include "common.cuh"
#include "det_util.cuh"

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
struct geometry_kernel_args {
  const T* r;
  const T* R;
  const int* pair_ij;
  int64_t Bc;
  int N;
  int M;
  int n_ee;
  int E;
  int Q;
  int ej;
  double rc;
  T* geo;
  T* rbf;
};

template <class T>
__device__ __forceinline__ void geometry_kernel_body(const int64_t bx_, const int by_, const int64_t nbx_, const T* __restrict__ r, const T* __restrict__ R, const int* __restrict__ pair_ij,
                                int64_t Bc, int N, int M, int n_ee, int E, int Q, int ej, double rc,
                                T* __restrict__ geo, T* __restrict__ rbf) {
  const int64_t gid = (int64_t)bx_ * blockDim.x + threadIdx.x;
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

// One launch over several molecules: block b runs entry m of the table.
template <class T>
__global__ void geometry_kernel_group(const __grid_constant__ Grp<geometry_kernel_args<T>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  GRP_STATIC(m_, const auto& a_ = g.a[K_];
             geometry_kernel_body<T>(grp_bx(g, K_, l_), grp_by(g, K_, l_), g.nbx[K_], a_.r, a_.R, a_.pair_ij, a_.Bc, a_.N, a_.M, a_.n_ee, a_.E, a_.Q, a_.ej, a_.rc, a_.geo, a_.rbf);)
}

// Edge hidden layer a = tanh(W1 e + b1) as a jet in d: (a, a', a'').
// W1 and b1 of the three edge types are staged in shared memory once per CTA
// ([t][q][a]); the persistent CTAs then stream blocks of kEdgesPerCta
// consecutive (walker, edge) rows.  A thread computes kHiddenVec consecutive
// features of one edge (vector loads of W1, vector stores), so D / kHiddenVec
// threads cover an edge and one warp holds one edge type.
constexpr int kEdgesPerCta = 32;
constexpr int kHiddenThreads = 256;

template <class T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};

template <class T>
struct edge_hidden_kernel_args {
  const T* rbf;
  const T* params;
  int64_t Bc;
  int E;
  int n_par;
  int n_ee;
  int D;
  int Q;
  int ej;
  int64_t W1_0;
  int64_t W1_1;
  int64_t W1_2;
  int64_t b1_0;
  int64_t b1_1;
  int64_t b1_2;
  T* eh;
};

template <class T>
__device__ __forceinline__ void edge_hidden_kernel_body(const int64_t bx_, const int by_, const int64_t nbx_, const T* __restrict__ rbf, const T* __restrict__ params, int64_t Bc, int E, int n_par,
                       int n_ee, int D, int Q, int ej, int64_t W1_0, int64_t W1_1, int64_t W1_2, int64_t b1_0,
                       int64_t b1_1, int64_t b1_2, T* __restrict__ eh) {
  using V = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ws = reinterpret_cast<T*>(smem_raw);  // [3][Q][D]
  T* bs = Ws + 3 * Q * D;                  // [3][D]
  T* fs = bs + 3 * D;                      // [kEdgesPerCta][ej][Q] features of this block's rows
  const int64_t W1o[3] = {W1_0, W1_1, W1_2}, b1o[3] = {b1_0, b1_1, b1_2};
  for (int t = 0; t < 3; ++t)
    for (int a = threadIdx.x; a < D; a += blockDim.x) {
      const T* src = params + W1o[t] + (int64_t)a * Q;
      for (int q = 0; q < Q; ++q) Ws[(t * Q + q) * D + a] = src[q];
      bs[t * D + a] = params[b1o[t] + a];
    }
  const int tpe = D / VW;                        // threads per edge
  const int epp = blockDim.x / tpe;              // edges in parallel
  const int er = threadIdx.x / tpe, a0 = (threadIdx.x % tpe) * VW;
  const int64_t nrows = Bc * E;
  for (int64_t be0 = (int64_t)bx_ * kEdgesPerCta; be0 < nrows; be0 += (int64_t)nbx_ * kEdgesPerCta) {
    const int nb = (int)min((int64_t)kEdgesPerCta, nrows - be0);
    __syncthreads();  // previous block's features consumed (and the weights staged)
    for (int k = threadIdx.x; k < nb * ej * Q; k += blockDim.x) fs[k] = rbf[be0 * ej * Q + k];
    __syncthreads();
    if (er >= epp) continue;
    auto type_of = [&](int r) {
      const int e = (int)((be0 + r) % E);
      return e < n_par ? 0 : (e < n_ee ? 1 : 2);
    };
    // NE consecutive edges of one type: every W1 load from shared memory serves NE edges
    auto rows = [&](auto ne, int r) {
      constexpr int NE = decltype(ne)::value;
      const int t = type_of(r);
      const T* W = Ws + t * Q * D + a0;
      T h[NE][VW], h1[NE][VW], h2[NE][VW];
      const V bv = *reinterpret_cast<const V*>(bs + t * D + a0);
      const T* bp = reinterpret_cast<const T*>(&bv);
#pragma unroll
      for (int n = 0; n < NE; ++n)
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          h[n][v] = bp[v];
          h1[n][v] = 0;
          h2[n][v] = 0;
        }
#pragma unroll 4
      for (int q = 0; q < Q; ++q) {
        const V wv = *reinterpret_cast<const V*>(W + q * D);
        const T* w = reinterpret_cast<const T*>(&wv);
#pragma unroll
        for (int n = 0; n < NE; ++n) {
          const T* f = fs + (r + n) * ej * Q;
          const T f0 = f[q];
#pragma unroll
          for (int v = 0; v < VW; ++v) h[n][v] += w[v] * f0;
          if (ej == 3) {
            const T f1 = f[Q + q], f2 = f[2 * Q + q];
#pragma unroll
            for (int v = 0; v < VW; ++v) {
              h1[n][v] += w[v] * f1;
              h2[n][v] += w[v] * f2;
            }
          }
        }
      }
#pragma unroll
      for (int n = 0; n < NE; ++n) {
        V o0, o1, o2;
        T* p0 = reinterpret_cast<T*>(&o0);
        T* p1 = reinterpret_cast<T*>(&o1);
        T* p2 = reinterpret_cast<T*>(&o2);
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          const T av = tanh_t(h[n][v]);
          p0[v] = av;
          const T da = T(1) - av * av;
          p1[v] = da * h1[n][v];
          p2[v] = da * h2[n][v] - T(2) * av * da * h1[n][v] * h1[n][v];
        }
        T* o = eh + (be0 + r + n) * ej * D + a0;
        *reinterpret_cast<V*>(o) = o0;
        if (ej == 3) {
          *reinterpret_cast<V*>(o + D) = o1;
          *reinterpret_cast<V*>(o + 2 * D) = o2;
        }
      }
    };
    auto pair = [&](int r) {  // edges r, r + 1 (if present)
      if (r + 1 < nb && type_of(r) == type_of(r + 1)) {
        rows(std::integral_constant<int, 2>{}, r);
      } else {
        rows(std::integral_constant<int, 1>{}, r);
        if (r + 1 < nb) rows(std::integral_constant<int, 1>{}, r + 1);
      }
    };
    if (ej == 1) {  // value rows: four edges per W1 load (registers allow it)
      for (int r = 4 * er; r < nb; r += 4 * epp) {
        const int t = type_of(r);
        if (r + 3 < nb && type_of(r + 1) == t && type_of(r + 2) == t && type_of(r + 3) == t) {
          rows(std::integral_constant<int, 4>{}, r);
        } else {
          pair(r);
          if (r + 2 < nb) pair(r + 2);
        }
      }
    } else {
      for (int r = 2 * er; r < nb; r += 2 * epp) pair(r);
    }
  }
}

// One launch over several molecules: block b runs entry m of the table.
template <class T>
__global__ void __launch_bounds__(kHiddenThreads) edge_hidden_kernel_group(const __grid_constant__ Grp<edge_hidden_kernel_args<T>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  GRP_STATIC(m_, const auto& a_ = g.a[K_];
             edge_hidden_kernel_body<T>(grp_bx(g, K_, l_), grp_by(g, K_, l_), g.nbx[K_], a_.rbf, a_.params, a_.Bc, a_.E, a_.n_par, a_.n_ee, a_.D, a_.Q, a_.ej, a_.W1_0, a_.W1_1, a_.W1_2, a_.b1_0, a_.b1_1, a_.b1_2, a_.eh);)
}

// ---------------------------------------------------------------------------
// Iterated edge embeddings (Eq. 16, second case): before the filters of layer
// l >= 1, f^l = f^{l-1} + tanh(U^{l,t} f^{l-1} + c^{l,t}) per edge type t, as
// a univariate jet in the edge's distance (value, d/dd, d2/dd2):
//   a = U f + c,  a' = U f',  a'' = U f'';  th = tanh a,  g = 1 - th^2;
//   f^l = f + th,  f^l' = f' + g a',  f^l'' = f'' + g a'' - 2 th g a'^2.
// One thread per (edge row, feature q); the rows of an iteration are staged
// in shared memory before any is written, so src may equal dst.
// ---------------------------------------------------------------------------
template <class T>
struct edge_update_kernel_args {
  const T* src;
  T* dst;
  const T* params;
  int64_t Bc;
  int E;
  int n_par;
  int n_ee;
  int Q;
  int ej;
  int64_t U0, U1, U2, c0, c1, c2;
};

template <class T>
__device__ __forceinline__ void edge_update_kernel_body(const int64_t bx_, const int64_t nbx_,
                                                        const edge_update_kernel_args<T>& a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Q = a.Q, ej = a.ej;
  T* Us = reinterpret_cast<T*>(smem_raw);  // [3][Q][Q]
  T* cs = Us + 3 * Q * Q;                  // [3][Q]
  T* fs = cs + 3 * Q;                      // [rows][ej][Q]
  const int64_t Uo[3] = {a.U0, a.U1, a.U2}, co[3] = {a.c0, a.c1, a.c2};
  for (int t = 0; t < 3; ++t) {
    for (int k = threadIdx.x; k < Q * Q; k += blockDim.x) Us[t * Q * Q + k] = a.params[Uo[t] + k];
    for (int k = threadIdx.x; k < Q; k += blockDim.x) cs[t * Q + k] = a.params[co[t] + k];
  }
  const int rpi = blockDim.x / Q;  // rows per iteration
  const int rr = threadIdx.x / Q, q = threadIdx.x % Q;
  const int64_t nrows = a.Bc * a.E;
  for (int64_t be0 = bx_ * rpi; be0 < nrows; be0 += nbx_ * rpi) {
    const int nb = (int)min((int64_t)rpi, nrows - be0);
    __syncthreads();  // weights staged; previous rows consumed
    for (int k = threadIdx.x; k < nb * ej * Q; k += blockDim.x) fs[k] = a.src[be0 * ej * Q + k];
    __syncthreads();
    if (rr >= nb) continue;
    const int64_t be = be0 + rr;
    const int e = (int)(be % a.E);
    const int t = e < a.n_par ? 0 : (e < a.n_ee ? 1 : 2);
    const T* f = fs + rr * ej * Q;
    const T* u = Us + (t * Q + q) * Q;
    T v = cs[t * Q + q], v1 = 0, v2 = 0;
    for (int k = 0; k < Q; ++k) {
      v += u[k] * f[k];
      if (ej == 3) {
        v1 += u[k] * f[Q + k];
        v2 += u[k] * f[2 * Q + k];
      }
    }
    const T th = tanh_t(v), g = T(1) - th * th;
    T* o = a.dst + be * ej * Q;
    o[q] = f[q] + th;
    if (ej == 3) {
      o[Q + q] = f[Q + q] + g * v1;
      o[2 * Q + q] = f[2 * Q + q] + g * v2 - T(2) * th * g * v1 * v1;
    }
  }
}

template <class T>
__global__ void __launch_bounds__(256) edge_update_kernel_group(const __grid_constant__ Grp<edge_update_kernel_args<T>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  GRP_STATIC(m_, edge_update_kernel_body<T>(grp_bx(g, K_, l_), g.nbx[K_], g.a[K_]);)
}

// ---------------------------------------------------------------------------
// Initial electron embeddings from the electron-nucleus difference vectors
// (Eq. 13, second case): x_i = (r_i - R_1, ..., r_i - R_M) and
// f^0_i = W_e2 tanh(W_e1 x_i + b_e1) + b_e2, with its jets in the coordinates.
// Only r_i moves x_i, and d x_i / d r_{i,c} = (e_c, ..., e_c); a = W_e1 x_i + b_e1
// is linear in r_i, so with h = tanh a, g = 1 - h^2 and u_c = sum_I W_e1[:, 3I + c]:
//   d h / d r_{i,c} = g u_c,   lap_i h = -2 h g sum_c u_c^2,
// and f^0 = W_e2 h + b_e2 channel by channel (value, the three channels of
// r_i, the Laplacian; every other channel is zero).  One thread per feature
// (blockDim = D), `per` electrons per CTA sharing each W_e2 load.
// ---------------------------------------------------------------------------
constexpr int kElInitMax = 8;
template <class T>
__global__ void __launch_bounds__(512)
    el_init_kernel(const T* __restrict__ r, const T* __restrict__ R, const T* __restrict__ params, int64_t W_e1,
                   int64_t b_e1, int64_t W_e2, int64_t b_e2, int64_t Bc, int N, int M, int D, int C, int per,
                   T* __restrict__ F, __nv_bfloat16* __restrict__ Fbf, T* __restrict__ H0, T* __restrict__ X0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M3 = 3 * M, nch = C > 1 ? 5 : 1;
  T* xs = reinterpret_cast<T*>(smem_raw);  // [per][3M]
  T* Hs = xs + per * M3;                   // [per][nch][D]
  const int a = threadIdx.x;
  const int64_t n_el = Bc * N, e0 = (int64_t)blockIdx.x * per;
  const int ne = (int)min((int64_t)per, n_el - e0);
  for (int k = a; k < ne * M3; k += blockDim.x) {
    const int e = k / M3, kk = k - e * M3, I = kk / 3, c = kk - I * 3;
    const T x = r[(e0 + e) * 3 + c] - R[I * 3 + c];
    xs[k] = x;
    if (X0) X0[(e0 + e) * M3 + kk] = x;
  }
  __syncthreads();
  const T* w1 = params + W_e1 + (int64_t)a * M3;
  T u0 = 0, u1 = 0, u2 = 0;
  for (int I = 0; I < M; ++I) {
    u0 += w1[3 * I];
    u1 += w1[3 * I + 1];
    u2 += w1[3 * I + 2];
  }
  const T usq = u0 * u0 + u1 * u1 + u2 * u2;
  for (int e = 0; e < ne; ++e) {
    T v = params[b_e1 + a];
    for (int k = 0; k < M3; ++k) v += w1[k] * xs[e * M3 + k];
    const T h = tanh_t(v), g = T(1) - h * h;
    T* hs = Hs + (e * nch) * D + a;
    hs[0] = h;
    if (nch == 5) {
      hs[D] = g * u0;
      hs[2 * D] = g * u1;
      hs[3 * D] = g * u2;
      hs[4 * D] = T(-2) * h * g * usq;
    }
    if (H0) H0[(e0 + e) * D + a] = h;
  }
  __syncthreads();
  T acc[kElInitMax][5];
#pragma unroll
  for (int e = 0; e < kElInitMax; ++e)
#pragma unroll
    for (int c = 0; c < 5; ++c) acc[e][c] = 0;
  const T* w2 = params + W_e2 + (int64_t)a * D;
  for (int k = 0; k < D; ++k) {
    const T w = w2[k];
#pragma unroll
    for (int e = 0; e < kElInitMax; ++e) {
      if (e >= ne) break;
      const T* hs = Hs + (e * nch) * D + k;
      acc[e][0] += w * hs[0];
      if (nch == 5) {
#pragma unroll
        for (int c = 1; c < 5; ++c) acc[e][c] += w * hs[c * D];
      }
    }
  }
  const T bias = params[b_e2 + a];
#pragma unroll
  for (int e = 0; e < kElInitMax; ++e) {
    if (e >= ne) break;
    const int64_t el = e0 + e;
    const int i = (int)(el % N);
    T* o = F + el * C * D + a;
    __nv_bfloat16* ob = Fbf ? Fbf + el * C * D + a : nullptr;
    for (int ch = 0; ch < C; ++ch) {
      T v = 0;
      if (ch == 0) v = acc[e][0] + bias;
      else if (ch == C - 1) v = acc[e][4];
      else if (ch >= 1 + 3 * i && ch < 4 + 3 * i) v = acc[e][ch - 3 * i];
      o[(int64_t)ch * D] = v;
      if (ob) ob[(int64_t)ch * D] = __float2bfloat16_rn((float)v);
    }
  }
}

// z0[s][a] = (W_h^0 E_spin[s])[a]: the node map of layer 0 on the spin embeddings.
template <class T>
struct layer0_node_kernel_args {
  const T* params;
  int D;
  int64_t E_spin;
  int64_t W_h;
  T* z0;
};

template <class T>
__device__ __forceinline__ void layer0_node_kernel_body(const int64_t bx_, const int by_, const int64_t nbx_, const T* __restrict__ params, int D, int64_t E_spin, int64_t W_h, T* z0) {
  const int gid = bx_ * blockDim.x + threadIdx.x;
  if (gid >= 2 * D) return;
  const int s = gid / D, a = gid % D;
  T acc = 0;
  for (int c = 0; c < D; ++c) acc += params[W_h + (int64_t)a * D + c] * params[E_spin + s * D + c];
  z0[gid] = acc;
}

// One launch over several molecules: block b runs entry m of the table.
template <class T>
__global__ void layer0_node_kernel_group(const __grid_constant__ Grp<layer0_node_kernel_args<T>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  GRP_STATIC(m_, const auto& a_ = g.a[K_];
             layer0_node_kernel_body<T>(grp_bx(g, K_, l_), grp_by(g, K_, l_), g.nbx[K_], a_.params, a_.D, a_.E_spin, a_.W_h, a_.z0);)
}

// ---------------------------------------------------------------------------
// Messages, Eq. (17), normalised per edge type, with the product rule.
//
// For every feature d the messages of channel c are two masked N x N
// matrices (same-spin / opposite-spin edge filters w_ij, zero diagonal)
// applied to the node channels z[j][c], plus the product-rule terms with
// derivatives of w_ij, which are nonzero only for the coordinates of i or j
// (u_ij = (r_i - r_j) / d_ij, w' and w'' the radial derivatives):
//  (a) channel of a SENDER's coordinate (c = 1 + 3e + x, e != i):
//      -w'_ie u_ie,x z_e[0];
//  (b) channel of the RECEIVER's own coordinate (c = 1 + 3i + x):
//      sum_j w'_ij u_ij,x z_j[0], and sum_I w'_iI u_iI,x Y_I for the nuclei;
//  (c) Laplacian channel: sum_j (2 w'' + 4 w'/d) z_j[0] + 2 w' u.(dz_j/dr_i - dz_j/dr_j),
//      and sum_I (w''_iI + 2 w'_iI / d_iI) Y_I;
//  (d) value channel: electron-nucleus messages sum_I w_iI Y_I.
//
// Jets: one CTA per (walker, chunk of 32 features), lanes over features.
// The filters are symmetric in (i, j), so w and w' are staged as N x N
// tables whose row j lists the receivers i: the IB receivers of a block sit
// at fixed offsets.  Signed unit vectors u_ij and z_j[0] are staged too.
// Phase 1 (all warps): the per-receiver terms (b), (c), (d) into shared
// memory.  Phase 2: a warp owns IB receivers x CB channels of one spin block
// and runs two passes (same-spin, opposite-spin senders) accumulating in
// registers, adds (a), then the phase-1 terms, and stores.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T to_out(float v, T*) { return (T)v; }
__device__ __forceinline__ double to_out(double v, double*) { return v; }
__device__ __forceinline__ __nv_bfloat16 to_out(float v, __nv_bfloat16*) { return __float2bfloat16_rn(v); }

constexpr int kMsgLanes = 32;

// Shared-memory layout of the jet message kernel (element offsets in T).
struct MsgSmem {
  int w0, w1, us, invd, z0c, zself, sp, ring, ps, total_bytes;
};
constexpr int kMsgRing = 4;     // senders in flight per warp (asynchronous copies)
constexpr int kMsgWarps = 8;
// L: features per CTA (lanes of a group; 32, or 16 for molecules whose pair
// tables do not fit at 32).
template <class T>
__host__ __device__ inline MsgSmem msg_smem_layout(int N, int IB, int CB, bool stage_w1, int L) {
  MsgSmem m{};
  int o = 0;
  const int rows = N * N + IB;  // padded: receivers past the end read zeros
  m.w0 = o; o += rows * L;
  m.w1 = o; o += stage_w1 ? rows * L : 0;
  m.us = o; o += (N + IB) * N * 3;  // u_ij,x (zero diagonal, zero padding)
  m.invd = o; o += N * N;
  m.z0c = o; o += N * L;       // z_j[0]
  m.zself = o; o += 3 * N * L;  // dz_j / dr_j,x
  m.sp = o; o += 13 * N * L;   // (b) [N][3 x][3], (c) [N][3], (d) [N]
  o = (o + 3) / 4 * 4;         // 16-byte alignment of the copy ring
  m.ring = o; o += kMsgWarps * 32 * kMsgRing * CB;  // [group][slot][q][lane] z of senders in flight
  m.ps = o * (int)sizeof(T);           // byte offset of the int pair table
  m.total_bytes = m.ps + N * N * (int)sizeof(int);
  return m;
}

template <class T, class TO>
struct messages_kernel_args {
  const T* Z;
  const T* z0;
  const T* ew;
  const T* geo;
  const T* Y;
  const int* pair_of;
  int N;
  int n_up;
  int M;
  int C;
  int D;
  int E;
  int n_ee;
  int z_const;
  int stage_w1;
  TO* msg;
};

template <class T, class TO, int IB, int CB, int L>
__device__ __forceinline__ void messages_kernel_body(const int64_t bx_, const int by_, const int64_t nbx_, const T* __restrict__ Z, const T* __restrict__ z0, const T* __restrict__ ew,
                    const T* __restrict__ geo, const T* __restrict__ Y, const int* __restrict__ pair_of, int N,
                    int n_up, int M, int C, int D, int E, int n_ee, int z_const, int stage_w1,
                    TO* __restrict__ msg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int ej = 3;
  const MsgSmem lay = msg_smem_layout<T>(N, IB, CB, stage_w1 != 0, L);
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* W0 = sm + lay.w0;  // [(j*N + i)][L]  w_ij
  T* W1 = sm + lay.w1;  //                 w'_ij
  T* Us = sm + lay.us;  // [(i*N + j)][3]
  T* Id = sm + lay.invd;
  T* Z0c = sm + lay.z0c;  // [j][L]
  T* Zsf = sm + lay.zself;  // [j][x][L]
  T* SP = sm + lay.sp;
  T* Ring = sm + lay.ring;
  int* Ps = reinterpret_cast<int*>(smem_raw + lay.ps);
  T* SPb = SP;               // [i][x][3]  (same, opposite, nucleus)
  T* SPc = SP + 9 * N * L;   // [i][3]
  T* SPd = SP + 12 * N * L;  // [i]

  const int64_t b = bx_;
  const int d0 = by_ * L;
  const int tid = threadIdx.x, lane = tid % L, grp = tid / L, ngroups = blockDim.x / L;
  const T* EWb = ew + b * E * ej * D + d0 + lane;  // this lane's feature of every edge filter
  const T* Zb = Z + b * N * C * D + d0 + lane;
  const T* Yd = Y + d0 + lane;
  const T* Gb = geo + b * E * 4;
  const int NN = N * N;

  // Pull this CTA's slices of the node channels and edge filters into L2.
  if (!z_const)
    for (int r = tid; r < N * C; r += blockDim.x)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(Z + (b * N * C + r) * D + d0));
  for (int r = tid; r < E * ej; r += blockDim.x)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ew + (b * E * ej + r) * D + d0));

  // ---- staging ----
  for (int k = tid; k < NN; k += blockDim.x) {
    const int i = k / N, j = k - (k / N) * N;
    const int p = pair_of[k];
    Ps[k] = p;
    T u0 = 0, u1 = 0, u2 = 0, id = 0;
    if (i != j) {
      const T sg = i < j ? T(1) : T(-1);
      u0 = sg * Gb[p * 4 + 1];
      u1 = sg * Gb[p * 4 + 2];
      u2 = sg * Gb[p * 4 + 3];
      id = T(1) / Gb[p * 4];
    }
    Us[k * 3] = u0;
    Us[k * 3 + 1] = u1;
    Us[k * 3 + 2] = u2;
    Id[k] = id;
  }
  for (int k = tid; k < IB * N * 3; k += blockDim.x) Us[NN * 3 + k] = T(0);
  TO* mb = msg + b * N * C * 3 * D + d0 + lane;
  // electron-nucleus part of every output: zero except in the value, Laplacian and
  // own-coordinate channels, which are written after phase 1
  for (int i = grp; i < N; i += ngroups) {
    TO* o = mb + (int64_t)i * C * 3 * D + 2 * D;
    for (int c = 0; c < C; ++c, o += 3 * D) *o = to_out(T(0), o);
  }
  __syncthreads();  // pair table ready
  // filter tables; rows are independent, so several loads are in flight per warp
#pragma unroll 4
  for (int r = grp; r < NN + IB; r += ngroups) {
    T v0 = 0, v1 = 0;
    const int p = r < NN ? Ps[r] : -1;  // Ps[j * N + i]: the edge (i, j), -1 on the diagonal
    if (p >= 0) {
      const T* w = EWb + (int64_t)p * ej * D;
      v0 = w[0];
      v1 = w[D];
    }
    W0[r * L + lane] = v0;
    if (stage_w1) W1[r * L + lane] = v1;
  }
  for (int j = grp; j < N; j += ngroups) {
    const T* zj = Zb + (int64_t)j * C * D;
    Z0c[j * L + lane] = z_const ? z0[(j < n_up ? 0 : D) + d0 + lane] : zj[0];
#pragma unroll
    for (int x = 0; x < 3; ++x) Zsf[(j * 3 + x) * L + lane] = z_const ? T(0) : zj[(int64_t)(1 + 3 * j + x) * D];
  }
  __syncthreads();
  // w' and w'' of the edge (i, j) for this lane (zero on the diagonal)
  auto w1_at = [&](int i, int j) -> T {
    if (stage_w1) return W1[(j * N + i) * L + lane];
    return i == j ? T(0) : EWb[((int64_t)Ps[i * N + j] * ej + 1) * D];
  };

  // ---- phase 1: per-receiver terms (b), (c), (d) ----
  // items: 3N of kind (b) (receiver, axis), 2N of kind (c) (receiver, sender spin), N of kind (d)
  const int n_dn = N - n_up;
  for (int it = grp; it < 6 * N; it += ngroups) {
    if (it < 3 * N) {  // (b) receiver i, axis x
      const int i = it / 3, x = it - (it / 3) * 3;
      const bool up = i < n_up;
      T sa = 0, sb = 0, sn = 0;  // spin up senders, spin down senders
#pragma unroll 4
      for (int j = 0; j < n_up; ++j) sa += w1_at(i, j) * Us[(i * N + j) * 3 + x] * Z0c[j * L + lane];
#pragma unroll 4
      for (int j = n_up; j < N; ++j) sb += w1_at(i, j) * Us[(i * N + j) * 3 + x] * Z0c[j * L + lane];
      for (int I = 0; I < M; ++I) {
        const int en = i * M + I;
        sn += EWb[((int64_t)(n_ee + en) * ej + 1) * D] * Gb[(n_ee + en) * 4 + 1 + x] * Yd[(int64_t)I * D];
      }
      T* o = SPb + (i * 3 + x) * 3 * L + lane;
      o[0] = up ? sa : sb;
      o[L] = up ? sb : sa;
      o[2 * L] = sn;
    } else if (it < 5 * N) {  // (c) Laplacian channel of receiver i, senders of one spin
      const int i = (it - 3 * N) >> 1, h = (it - 3 * N) & 1;
      const bool up = i < n_up;
      const int j0 = h == 0 ? 0 : n_up, j1 = h == 0 ? n_up : N;
      const T* zc = Zb + (int64_t)(1 + 3 * i) * D;  // dz_j / dr_i of sender j at zc + j * C * D
      T sv = 0;
      // senders in batches of kCJ: every global load of a batch (w'' and the three channels
      // dz_j / dr_i) is issued before any is used, so their latencies overlap
      constexpr int kCJ = 8;
      for (int jb = j0; jb < j1; jb += kCJ) {
        T w2v[kCJ], zx[kCJ], zy[kCJ], zz[kCJ];
#pragma unroll
        for (int u = 0; u < kCJ; ++u) {
          const int j = jb + u;
          const bool ok = j < j1 && j != i;
          w2v[u] = ok ? EWb[((int64_t)Ps[i * N + j] * ej + 2) * D] : T(0);
          const T* zj = zc + (int64_t)(ok ? j : i) * C * D;
          zx[u] = ok && !z_const ? zj[0] : T(0);
          zy[u] = ok && !z_const ? zj[D] : T(0);
          zz[u] = ok && !z_const ? zj[2 * D] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kCJ; ++u) {
          const int j = jb + u;
          if (j >= j1) break;
          const T v1 = w1_at(i, j);
          T t = (T(2) * w2v[u] + T(4) * v1 * Id[i * N + j]) * Z0c[j * L + lane];
          if (!z_const) {
            const T* uu = Us + (i * N + j) * 3;
            const T cr = uu[0] * (zx[u] - Zsf[(j * 3) * L + lane]) + uu[1] * (zy[u] - Zsf[(j * 3 + 1) * L + lane]) +
                         uu[2] * (zz[u] - Zsf[(j * 3 + 2) * L + lane]);
            t += T(2) * v1 * cr;
          }
          sv += t;
        }
      }
      SPc[(i * 3 + (up == (h == 0) ? 0 : 1)) * L + lane] = sv;
      if (h == 0) {
        T sn = 0;
        for (int I = 0; I < M; ++I) {
          const int en = i * M + I;
          const T* w = EWb + (int64_t)(n_ee + en) * ej * D;
          sn += (w[2 * D] + T(2) * w[D] / Gb[(n_ee + en) * 4]) * Yd[(int64_t)I * D];
        }
        SPc[(i * 3 + 2) * L + lane] = sn;
      }
    } else {  // (d) value channel, nuclei
      const int i = it - 5 * N;
      T sn = 0;
      for (int I = 0; I < M; ++I) sn += EWb[(int64_t)(n_ee + i * M + I) * ej * D] * Yd[(int64_t)I * D];
      SPd[i * L + lane] = sn;
    }
  }
  __syncthreads();

  // electron-nucleus part of the value, Laplacian and own-coordinate channels
  const T nuM = T(1) / T(M);
  for (int k = grp; k < 5 * N; k += ngroups) {
    const int i = k / 5, kind = k - (k / 5) * 5;
    const int c = kind == 0 ? 0 : (kind == 1 ? C - 1 : 1 + 3 * i + (kind - 2));
    const T v = kind == 0 ? SPd[i * L + lane]
                          : (kind == 1 ? SPc[(i * 3 + 2) * L + lane] : SPb[((i * 3 + kind - 2) * 3 + 2) * L + lane]);
    TO* o = mb + ((int64_t)i * C + c) * 3 * D + 2 * D;
    *o = to_out(v * nuM, o);
  }

  // ---- phase 2: main contraction ----
  const int nib_up = (n_up + IB - 1) / IB, nib_dn = (n_dn + IB - 1) / IB;
  const int ncb = (C + CB - 1) / CB;
  const int ntasks = (nib_up + nib_dn) * ncb;
  const int CD = C * D;
  for (int task = grp; task < ntasks; task += ngroups) {
    const int ibk = task / ncb, cbk = task - (task / ncb) * ncb;
    const bool up = ibk < nib_up;
    const int sb0 = up ? 0 : n_up, sbn = up ? n_up : n_dn;  // spin block of the receivers
    const int i0 = sb0 + (up ? ibk : ibk - nib_up) * IB;
    const int ni = min(IB, sb0 + sbn - i0);
    const int c0 = cbk * CB;
    const int nc = min(CB, C - c0);
    const int os0 = up ? n_up : 0, osn = up ? n_dn : n_up;  // opposite spin block (senders)
    const int qlap = c0 + nc == C ? C - 1 - c0 : -1;
    int eq[CB], xq[CB];  // electron / axis of the coordinate channels (-1: none)
#pragma unroll
    for (int q = 0; q < CB; ++q) {
      const int c = c0 + q;
      const bool coord = q < nc && c >= 1 && c < C - 1;
      eq[q] = coord ? (c - 1) / 3 : -1;
      xq[q] = coord ? (c - 1) - ((c - 1) / 3) * 3 : 0;
    }
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      const int j0 = pass == 0 ? sb0 : os0, jn = pass == 0 ? sbn : osn;
      T acc[IB][CB];
#pragma unroll
      for (int a = 0; a < IB; ++a)
#pragma unroll
        for (int q = 0; q < CB; ++q) acc[a][q] = T(0);
      if (z_const && c0 == 0) {  // constant z: only the value channel, z_j[0] staged
        const T* wp = W0 + (j0 * N + i0) * L + lane;
#pragma unroll 1
        for (int jj = 0; jj < jn; ++jj, wp += N * L) {
          const T z = Z0c[(j0 + jj) * L + lane];
#pragma unroll
          for (int a = 0; a < IB; ++a) acc[a][0] += wp[a * L] * z;
        }
      } else if (!z_const && jn > 0) {
        // z_j[c0 .. c0 + CB) of the next kMsgRing senders in flight as asynchronous
        // copies into this warp's ring; each lane copies and later reads its own feature.
        const T* zp = Zb + (int64_t)j0 * CD + c0 * D;
        const uint32_t ring = (uint32_t)__cvta_generic_to_shared(Ring + grp * kMsgRing * CB * L + lane);
        auto issue = [&](int jj) {
          if (jj < jn) {
            const T* src = zp + (int64_t)jj * CD;
            const uint32_t dst = ring + (uint32_t)((jj % kMsgRing) * CB * L * sizeof(T));
#pragma unroll
            for (int q = 0; q < CB; ++q)
              if (q < nc)
                asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst + (uint32_t)(q * L * sizeof(T))),
                             "l"(src + (int64_t)q * D), "n"(sizeof(T))
                             : "memory");
          }
          asm volatile("cp.async.commit_group;" ::: "memory");
        };
#pragma unroll
        for (int u = 0; u < kMsgRing; ++u) issue(u);
        const T* wp = W0 + (j0 * N + i0) * L + lane;
        const T* rs = Ring + grp * kMsgRing * CB * L + lane;
#pragma unroll 1
        for (int jj = 0; jj < jn; ++jj, wp += N * L) {
          asm volatile("cp.async.wait_group %0;" ::"n"(kMsgRing - 1) : "memory");
          T zc[CB];
          const T* slot = rs + (jj % kMsgRing) * CB * L;
#pragma unroll
          for (int q = 0; q < CB; ++q) zc[q] = q < nc ? slot[q * L] : T(0);
#pragma unroll
          for (int a = 0; a < IB; ++a) {
            const T w = wp[a * L];
#pragma unroll
            for (int q = 0; q < CB; ++q) acc[a][q] += w * zc[q];
          }
          issue(jj + kMsgRing);  // refill the slot just consumed
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
#pragma unroll
      for (int q = 0; q < CB; ++q) {
        const int e = eq[q];
        // (a): the channel holds a coordinate of a sender of this pass
        if (e >= j0 && e < j0 + jn) {
          const T ze0 = Z0c[e * L + lane];
          const T* ue = Us + (i0 * N + e) * 3 + xq[q];
#pragma unroll
          for (int a = 0; a < IB; ++a)
            if (a < ni) acc[a][q] -= w1_at(i0 + a, e) * ue[a * N * 3] * ze0;
        }
        // (b): the channel holds a coordinate of a receiver of this block
        if (e >= i0 && e < i0 + ni) {
          const T v = SPb[((e * 3 + xq[q]) * 3 + pass) * L + lane];
#pragma unroll
          for (int a = 0; a < IB; ++a)
            if (i0 + a == e) acc[a][q] += v;
        }
        // (c): Laplacian channel
        if (q == qlap) {
#pragma unroll
          for (int a = 0; a < IB; ++a)
            if (a < ni) acc[a][q] += SPc[((i0 + a) * 3 + pass) * L + lane];
        }
      }
      const T nu = T(1) / T(pass == 0 ? (sbn - 1 > 1 ? sbn - 1 : 1) : (osn > 1 ? osn : 1));
      TO* ob = mb + ((int64_t)i0 * C + c0) * 3 * D + pass * D;
#pragma unroll
      for (int a = 0; a < IB; ++a) {
        if (a >= ni) continue;
#pragma unroll
        for (int q = 0; q < CB; ++q) {
          if (q >= nc) continue;
          TO* o = ob + ((int64_t)a * C + q) * 3 * D;
          *o = to_out(acc[a][q] * nu, o);
        }
      }
    }
  }
}

// One launch over several molecules: block b runs entry m of the table; the
// entry's tag is its features per CTA (32, or 16 for large molecules).
template <class T, class TO, int IB, int CB>
__global__ void __launch_bounds__(256, 2) messages_kernel_group(const __grid_constant__ Grp<messages_kernel_args<T, TO>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  const messages_kernel_args<T, TO>& a_ = g.a[m_];
  if (g.tag[m_] == 16)
    messages_kernel_body<T, TO, IB, CB, 16>(grp_bx(g, m_, l_), grp_by(g, m_, l_), g.nbx[m_], a_.Z, a_.z0, a_.ew, a_.geo,
                                            a_.Y, a_.pair_of, a_.N, a_.n_up, a_.M, a_.C, a_.D, a_.E, a_.n_ee,
                                            a_.z_const, a_.stage_w1, a_.msg);
  else
    messages_kernel_body<T, TO, IB, CB, kMsgLanes>(grp_bx(g, m_, l_), grp_by(g, m_, l_), g.nbx[m_], a_.Z, a_.z0, a_.ew,
                                                   a_.geo, a_.Y, a_.pair_of, a_.N, a_.n_up, a_.M, a_.C, a_.D, a_.E,
                                                   a_.n_ee, a_.z_const, a_.stage_w1, a_.msg);
}

// Value-only messages (C = 1): one CTA per (walker, 32 features); a warp per
// receiver, lanes over features; pair table and z of the walker staged in
// shared memory, sender loops split by spin (no per-edge branch).
template <class T, class TO>
struct messages_value_kernel_args {
  const T* Z;
  const T* z0;
  const T* ew;
  const T* Y;
  const int* pair_of;
  int64_t Bc;
  int N;
  int n_up;
  int M;
  int D;
  int E;
  int n_ee;
  int z_const;
  TO* msg;
};

template <class T, class TO>
__device__ __forceinline__ void messages_value_kernel_body(const int64_t bx_, const int by_, const int64_t nbx_, const T* __restrict__ Z, const T* __restrict__ z0, const T* __restrict__ ew,
                          const T* __restrict__ Y, const int* __restrict__ pair_of, int64_t Bc, int N, int n_up,
                          int M, int D, int E, int n_ee, int z_const, TO* __restrict__ msg) {
  extern __shared__ __align__(16) unsigned char mv_smem[];
  T* Zs = reinterpret_cast<T*>(mv_smem);           // [N][32]
  int* Ps = reinterpret_cast<int*>(Zs + N * 32);   // [N][N]
  const int64_t b = bx_;
  const int lane = threadIdx.x % 32, wq = threadIdx.x / 32, nw = blockDim.x / 32;
  const int d = by_ * 32 + lane;
  for (int k = threadIdx.x; k < N * N; k += blockDim.x) Ps[k] = pair_of[k];
  for (int j = wq; j < N; j += nw)
    Zs[j * 32 + lane] = d >= D ? T(0) : (z_const ? z0[(j < n_up ? 0 : D) + d] : Z[(b * N + j) * D + d]);
  __syncthreads();
  if (d >= D) return;
  const T* ewb = ew + b * E * D + d;
  for (int i = wq; i < N; i += nw) {
    const bool up = i < n_up;
    T su = 0, sd = 0, sn = 0;  // spin-up senders, spin-down senders, nuclei
#pragma unroll 4
    for (int j = 0; j < n_up; ++j)
      if (j != i) su += ewb[(int64_t)Ps[i * N + j] * D] * Zs[j * 32 + lane];
#pragma unroll 4
    for (int j = n_up; j < N; ++j)
      if (j != i) sd += ewb[(int64_t)Ps[i * N + j] * D] * Zs[j * 32 + lane];
    for (int I = 0; I < M; ++I) sn += ewb[(int64_t)(n_ee + i * M + I) * D] * Y[(int64_t)I * D + d];
    const int n_same = up ? n_up : N - n_up, n_opp = N - n_same;
    TO* out = msg + (b * N + i) * 3 * D + d;
    out[0] = to_out((up ? su : sd) / T(n_same - 1 > 1 ? n_same - 1 : 1), out);
    out[D] = to_out((up ? sd : su) / T(n_opp > 1 ? n_opp : 1), out);
    out[2 * D] = to_out(sn / T(M), out);
  }
}

// One launch over several molecules: block b runs entry m of the table.
template <class T, class TO>
__global__ void __launch_bounds__(256) messages_value_kernel_group(const __grid_constant__ Grp<messages_value_kernel_args<T, TO>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  const messages_value_kernel_args<T, TO>& a_ = g.a[m_];
  messages_value_kernel_body<T, TO>(grp_bx(g, m_, l_), grp_by(g, m_, l_), g.nbx[m_], a_.Z, a_.z0, a_.ew, a_.Y, a_.pair_of, a_.Bc, a_.N, a_.n_up, a_.M, a_.D, a_.E, a_.n_ee, a_.z_const, a_.msg);
}

// ---------------------------------------------------------------------------
// Residual tanh update, Eq. (18): f <- f + tanh(P) with jets.
// ---------------------------------------------------------------------------
template <class T>
struct update_kernel_args {
  const T* P;
  const T* Fin;
  T* Fout;
  const T* E_spin;
  int64_t Bc;
  int N;
  int n_up;
  int C;
  int D;
  int from_spin;
  __nv_bfloat16* Fbf;
};

template <class T>
__device__ __forceinline__ void update_kernel_body(const int64_t bx_, const int by_, const int64_t nbx_, const T* __restrict__ P, const T* Fin, T* Fout, const T* __restrict__ E_spin,
                              int64_t Bc, int N, int n_up, int C, int D, int from_spin,
                              __nv_bfloat16* __restrict__ Fbf) {
  const int64_t gid = (int64_t)bx_ * blockDim.x + threadIdx.x;
  if (gid >= Bc * N * D) return;
  const int a = (int)(gid % D);
  const int64_t bi = gid / D;
  const int i = (int)(bi % N);
  const T* p = P + bi * C * D + a;
  const T* fi = Fin + bi * C * D + a;
  T* f = Fout + bi * C * D + a;
  const T t = tanh_t(p[0]);
  const T dt = T(1) - t * t;
  f[0] = (from_spin ? E_spin[(i < n_up ? 0 : 1) * D + a] : fi[0]) + t;
  if (C > 1) {
    T ss = 0;
    for (int c = 1; c < C - 1; ++c) {
      const T pc = p[(int64_t)c * D];
      ss += pc * pc;
      f[(int64_t)c * D] = (from_spin ? T(0) : fi[(int64_t)c * D]) + dt * pc;
    }
    const int64_t cl = (int64_t)(C - 1) * D;
    f[cl] = (from_spin ? T(0) : fi[cl]) + dt * p[cl] - T(2) * t * dt * ss;
  }
  if (Fbf) {  // BF16 copy of the embeddings: the input of the next node-map GEMM
    __nv_bfloat16* fb = Fbf + bi * C * D + a;
    for (int c = 0; c < C; ++c) fb[(int64_t)c * D] = __float2bfloat16_rn((float)f[(int64_t)c * D]);
  }
}

template <class T>
__global__ void update_kernel(const T* __restrict__ P, const T* Fin, T* Fout, const T* __restrict__ E_spin,
                              int64_t Bc, int N, int n_up, int C, int D, int from_spin,
                              __nv_bfloat16* __restrict__ Fbf) {
  update_kernel_body<T>(blockIdx.x, blockIdx.y, gridDim.x, P, Fin, Fout, E_spin, Bc, N, n_up, C, D, from_spin, Fbf);
}

// One launch over several molecules: block b runs entry m of the table.
template <class T>
__global__ void update_kernel_group(const __grid_constant__ Grp<update_kernel_args<T>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  GRP_STATIC(m_, const auto& a_ = g.a[K_];
             update_kernel_body<T>(grp_bx(g, K_, l_), grp_by(g, K_, l_), g.nbx[K_], a_.P, a_.Fin, a_.Fout, a_.E_spin, a_.Bc, a_.N, a_.n_up, a_.C, a_.D, a_.from_spin, a_.Fbf);)
}

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) dst[e] = __float2bfloat16_rn(src[e]);
}

// ---------------------------------------------------------------------------
// Orbitals x envelopes and determinant jets.  One warp per (walker, spin, p).
//
// Value-only calls (ansatz_eval, Metropolis) in FP32 mode factorise every
// matrix in FP32 first (LU with warp-level partial pivoting).  A condition
// estimate of the row-equilibrated matrix, kappa = n max_{k,i} |(A^-1)_ki| r_i
// with r_i = max_k |A_ik| (row scaling by the envelopes does not hurt the
// pivoted LU), decides whether that is accurate enough: near-nodal matrices
// (kappa above the threshold) are redone in FP64.  The local-energy path
// needs the determinant derivatives (tangent contractions with A^-1), whose
// plain FP32 rounding doubles the error of E_loc at near-nodal walkers: the
// FP32 jet bodies below (blocks of up to 28 electrons) refine the FP32
// inverse to a double-float pair and contract the tangents in double-float
// arithmetic on the FP32 pipes, because FP64 instructions issue at a small
// fraction of the FP32 rate on this GPU; the general body here takes FP64 for
// larger blocks.  In FP64 mode every step is FP64.
// ---------------------------------------------------------------------------
#ifndef DQ_KAPPA_FP32_VALUE
#define DQ_KAPPA_FP32_VALUE 10000.0f  // value-only log|det| in FP32 (corrected) below this
#endif

// Determinant derivatives: for every tangent t (3N coordinates, then the
// Laplacian channel) build d_t A into tmp and accumulate
// grad[t] = tr(A^-1 d_t A) and lap = tr(A^-1 L A) - sum_t tr((A^-1 d_t A)^2)
// in arithmetic S.
template <class T, class S>
__device__ double det_tangents(const T* phib, const T* env, const T* jenv, const T* lenv, const T* phi0, const S* Ainv,
                               S* tmp, S* X, int n, int nn, int i0, int p, int C, int Wo, int N3, int lane,
                               double* out) {
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
      tmp[q] = (S)v;
    }
    __syncwarp();
    S trp = 0;
    for (int q = lane; q < n * n; q += 32) {
      const int a = q / n, m = q % n;
      S x = 0;
      for (int l = 0; l < n; ++l) x += Ainv[a * n + l] * tmp[l * n + m];
      X[q] = x;
      if (a == m) trp += x;
    }
    const double tr = warp_sum((double)trp);
    __syncwarp();
    if (is_lap) {
      lap += tr;
    } else {
      if (lane == 0) out[2 + t] = tr;
      S s2 = 0;
      for (int q = lane; q < n * n; q += 32) {
        const int a = q / n, m = q % n;
        s2 += X[a * n + m] * X[m * n + a];
      }
      lap -= warp_sum((double)s2);
    }
    __syncwarp();
  }
  return lap;
}


// Determinant derivatives in double-float: A^-1 = Ahi + Alo (split from the
// FP64 inverse), d_t A exact in FP32 (it comes from the FP32 network), each
// entry of X = A^-1 d_t A a compensated dot product; tr X and tr X^2 in
// double-float.  Same quantities as det_tangents, on the FP32 pipes.
template <class T>
__device__ double det_tangents_df(const T* phib, const T* env, const T* jenv, const T* lenv, const T* phi0,
                                  const float* Ahi, const float* Alo, float* tmp, float* Xhi, float* Xlo, int n,
                                  int nn, int i0, int p, int C, int Wo, int N3, int lane, double* out) {
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
      tmp[q] = (float)v;
    }
    __syncwarp();
    dfloat trp = {0.f, 0.f};
    for (int q = lane; q < n * n; q += 32) {
      const int a = q / n, m = q % n;
      float sh = 0.f, cl = 0.f;
      for (int l = 0; l < n; ++l) {
        const float y = tmp[l * n + m], xh = Ahi[a * n + l];
        const float pr = __fmul_rn(xh, y);
        const float ep = __fmaf_rn(xh, y, -pr);
        const dfloat ss = two_sum(sh, pr);
        sh = ss.hi;
        cl = __fmaf_rn(Alo[a * n + l], y, __fadd_rn(cl, __fadd_rn(ep, ss.lo)));
      }
      const dfloat x = quick_two_sum(sh, cl);
      Xhi[q] = x.hi;
      Xlo[q] = x.lo;
      if (a == m) trp = df_add(trp, x);
    }
    const dfloat trs = warp_sum_df(trp);
    const double tr = (double)trs.hi + (double)trs.lo;
    __syncwarp();
    if (is_lap) {
      lap += tr;
    } else {
      if (lane == 0) out[2 + t] = tr;
      dfloat s2 = {0.f, 0.f};
      for (int q = lane; q < n * n; q += 32) {
        const int a = q / n, m = q % n;
        s2 = df_add(s2, df_mul({Xhi[a * n + m], Xlo[a * n + m]}, {Xhi[m * n + a], Xlo[m * n + a]}));
      }
      const dfloat s2s = warp_sum_df(s2);
      lap -= (double)s2s.hi + (double)s2s.lo;
    }
    __syncwarp();
  }
  return lap;
}

template <class T>
struct orbital_det_kernel_args {
  const T* phi;
  const T* geo;
  const T* params;
  int64_t Bc;
  int N;
  int n_up;
  int M;
  int K;
  int C;
  int Wo;
  int E;
  int n_ee;
  int64_t om_up;
  int64_t om_dn;
  int64_t ze_up;
  int64_t ze_dn;
  double* det;
  unsigned long long* n_fp64;
  int full;  // 1: block 0 is the N x N determinant of Eq. (22), block 1 the empty one
};

// Determinant blocks.  Every (walker, p) has two: the spin-up and spin-down
// matrices of Eq. (21), or (full) the N x N matrix of Eq. (22) and an empty
// block (determinant 1), so that the combination downstream is the same.
// Row ii of block s is electron i0 + ii; its orbitals and envelopes are those
// of the electron's own spin.
__device__ __forceinline__ void det_block(int s, int N, int n_up, int full, int& n, int& i0) {
  n = full ? (s == 0 ? N : 0) : (s == 0 ? n_up : N - n_up);
  i0 = (full || s == 0) ? 0 : n_up;
}

template <class T>
__device__ __forceinline__ void orbital_det_kernel_body(const int64_t bx_, const int by_, const int64_t nbx_, const T* __restrict__ phi, const T* __restrict__ geo, const T* __restrict__ params,
                       int64_t Bc, int N, int n_up, int M, int K, int C, int Wo, int E, int n_ee,
                       int64_t om_up, int64_t om_dn, int64_t ze_up, int64_t ze_dn, double* __restrict__ det,
                       unsigned long long* __restrict__ n_fp64, int full) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int warps = blockDim.x / 32;
  const int64_t gw = (int64_t)bx_ * warps + warp;
  const int n_dn = N - n_up;
  const int nmax = full ? N : (n_up > n_dn ? n_up : n_dn);
  const int N3 = 3 * N;
  const bool jets = C > 1;
  const int nn = nmax * nmax;
  const size_t per_warp = (size_t)nn * (3 * sizeof(double) + 10 * sizeof(T)) + 32 * sizeof(int);
  unsigned char* base = smem_raw + warp * ((per_warp + 15) / 16 * 16);
  double* LUd = reinterpret_cast<double*>(base);  // FP64 path
  double* Ainvd = LUd + nn;
  double* Xd = Ainvd + nn;
  T* env = reinterpret_cast<T*>(Xd + nn);
  T* jenv = env + nn;  // [3][nn]
  T* lenv = jenv + 3 * nn;
  T* phi0 = lenv + nn;
  T* LUt = phi0 + nn;  // arithmetic-type path
  T* Ainvt = LUt + nn;
  T* tmp = Ainvt + nn;
  T* Xt = tmp + nn;
  int* perm = reinterpret_cast<int*>(Xt + nn);

  if (gw >= Bc * 2 * K) return;
  const int64_t b = gw / (2 * K);
  const int s = (int)((gw / K) % 2);
  const int p = (int)(gw % K);
  int n, i0;
  det_block(s, N, n_up, full, n, i0);
  double* out = det + gw * (N3 + 3);
  if (n == 0) {  // empty determinant = 1
    for (int k = lane; k < N3 + 3; k += 32) out[k] = k == 0 ? 1.0 : 0.0;
    return;
  }
  const T* phib = phi + b * N * C * Wo;
  const T* gb = geo + b * E * 4;

  // Envelopes (Eq. 20) with their derivatives in the coordinates of electron i.
  T amax = 0;
  for (int q = lane; q < n * n; q += 32) {
    const int ii = q / n, k = q % n, o = p * n + k, i = i0 + ii;
    const bool up = i < n_up;
    const T* om = params + (up ? om_up : om_dn);
    const T* ze = params + (up ? ze_up : ze_dn);
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
    LUt[q] = f0 * ev;
    amax = max(amax, (T)fabs(f0 * ev));
  }
  __syncwarp();

  (void)amax;
  int sign = 0;
  double logabs = -INFINITY;
  bool fp64 = sizeof(T) == 8 || jets;
  if (!fp64) {
    T* rmax = Xt;  // row maxima of A (Xt is unused on the value-only path)
    if (lane < n) {
      T m = 0;
      for (int k = 0; k < n; ++k) m = max(m, (T)fabs(LUt[lane * n + k]));
      rmax[lane] = m;
    }
    __syncwarp();
    bool ok = warp_lu<T>(LUt, perm, n, lane, &sign, &logabs);
    if (ok) {
      warp_inverse<T>(LUt, perm, n, lane, Ainvt);
      T imax = 0;
      for (int q = lane; q < n * n; q += 32) imax = max(imax, (T)fabs(Ainvt[q]) * rmax[q % n]);
      const T kappa = T(n) * warp_max(imax);
      fp64 = !(kappa <= T(DQ_KAPPA_FP32_VALUE));
    } else {
      fp64 = true;
    }
    if constexpr (sizeof(T) == 4) {
      if (!fp64) {
        // log|det A| = log|det LU| + tr(A^-1 P^T (P A - L U)) to first order in the backward
        // error of the FP32 factorisation; entry (r, c) of P A - L U pairs with A^-1[c][perm[r]].
        float part = 0.f;
        for (int q = lane; q < n * n; q += 32) {
          const int r = q / n, c = q - (q / n) * n, mm = r < c ? r : c;
          const int ar = perm[r] * n + c;
          dfloat acc = {-(phi0[ar] * env[ar]), 0.f};
          for (int m = 0; m <= mm; ++m) acc = dot2_step(acc, m == r ? 1.f : LUt[r * n + m], LUt[m * n + c]);
          part = fmaf(Ainvt[c * n + perm[r]], -(acc.hi + acc.lo), part);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        logabs += (double)part;
      }
    }
  }
  if (fp64) {
    if (sizeof(T) == 4 && !jets && lane == 0) atomicAdd(n_fp64, 1ull);
    for (int q = lane; q < n * n; q += 32) LUd[q] = (double)phi0[q] * (double)env[q];
    __syncwarp();
    if (!warp_lu<double>(LUd, perm, n, lane, &sign, &logabs)) {
      for (int k = lane; k < N3 + 3; k += 32) out[k] = k == 1 ? -INFINITY : 0.0;
      return;
    }
  }
  if (lane == 0) {
    out[0] = (double)sign;
    out[1] = logabs;
  }
  if (!jets) return;
  double lap;
  warp_inverse<double>(LUd, perm, n, lane, Ainvd);
  if constexpr (sizeof(T) == 4) {
    // FP32 modes: tangent contractions in double-float on the FP32 pipes.
    float* Ahi = reinterpret_cast<float*>(LUt);
    float* Alo = reinterpret_cast<float*>(Ainvt);
    float* Xlo = reinterpret_cast<float*>(Xd);
    for (int q = lane; q < n * n; q += 32) {
      const double a = Ainvd[q];
      const float h = (float)a;
      Ahi[q] = h;
      Alo[q] = (float)(a - (double)h);
    }
    __syncwarp();
    lap = det_tangents_df<T>(phib, env, jenv, lenv, phi0, Ahi, Alo, reinterpret_cast<float*>(tmp),
                             reinterpret_cast<float*>(Xt), Xlo, n, nn, i0, p, C, Wo, N3, lane, out);
  } else {
    lap = det_tangents<T, double>(phib, env, jenv, lenv, phi0, Ainvd, LUd, Xd, n, nn, i0, p, C, Wo, N3, lane, out);
  }
  if (lane == 0) out[2 + N3] = lap;
}

template <class T>
__global__ void __launch_bounds__(128) orbital_det_kernel(const T* __restrict__ phi, const T* __restrict__ geo, const T* __restrict__ params,
                       int64_t Bc, int N, int n_up, int M, int K, int C, int Wo, int E, int n_ee,
                       int64_t om_up, int64_t om_dn, int64_t ze_up, int64_t ze_dn, double* __restrict__ det,
                       unsigned long long* __restrict__ n_fp64, int full) {
  orbital_det_kernel_body<T>(blockIdx.x, blockIdx.y, gridDim.x, phi, geo, params, Bc, N, n_up, M, K, C, Wo, E, n_ee, om_up, om_dn, ze_up, ze_dn, det, n_fp64, full);
}

// One launch over several molecules: block b runs entry m of the table.
template <class T>
__global__ void __launch_bounds__(128) orbital_det_kernel_group(const __grid_constant__ Grp<orbital_det_kernel_args<T>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  const orbital_det_kernel_args<T>& a_ = g.a[m_];
  orbital_det_kernel_body<T>(grp_bx(g, m_, l_), grp_by(g, m_, l_), g.nbx[m_], a_.phi, a_.geo, a_.params, a_.Bc, a_.N, a_.n_up, a_.M, a_.K, a_.C, a_.Wo, a_.E, a_.n_ee, a_.om_up, a_.om_dn, a_.ze_up, a_.ze_dn, a_.det, a_.n_fp64, a_.full);
}

// ---------------------------------------------------------------------------
// Determinant jets of the FP32 modes for spin blocks of at most kDetNR
// electrons, one warp per matrix, on the FP32 pipes:
//  * the factorisation of det_factor_jets below (FP32 LU, refined
//    double-float inverse Xhi + Xlo, log|det A| corrected for the backward
//    error of the FP32 LU; FP64 for ill-conditioned matrices, counted in n_fp64);
//  * the 3N + 1 tangents X_t = A^-1 d_t A as compensated dot products with
//    the rows of Xhi / Xlo in registers; tr X_t from the diagonal in
//    double-float, sum_t tr(X_t^2) accumulated per lane and reduced once.
// ---------------------------------------------------------------------------

// The factorisation step of the FP32 determinant jets (one warp, n <= 32):
//  * FP32 LU of A with partial pivoting and the inverse X0 from it; the
//    row-equilibrated condition estimate kappa = n max_ij |X0_ij| max_k |A_jk|;
//  * iterative refinement of the inverse as a double-float pair X = Xhi + Xlo,
//    X <- X + X (I - A X), with the residual as a compensated dot product
//    (Ogita-Rump-Oishi Dot2) over both parts of X; each step squares the
//    residual (of the order kappa u at the start), and the steps stop once the
//    largest residual entry before a step is at most 1e-4 (X then accurate to
//    about 1e-8 relative), at most four of them;
//  * log|det A| = log|det LU| - log det(I - E) with E = X (A - P^T L U) (exact
//    when X = A^-1), kept to second order: tr E + tr(E^2) / 2, with E of the
//    order kappa u (the third-order term is below 1e-5 up to DQ_KAPPA_FP32_JET_MAX);
//  * above DQ_KAPPA_FP32_JET_MAX, at a zero FP32 pivot, or when the refinement
//    does not converge, the FP64 LU and inverse instead, counted in n_fp64.
// rmax holds the row maxima of A; R and T are n x n scratch (not aliasing A, LU,
// X0, Xhi, Xlo or each other), LUd / Ainvd n x n doubles (may alias R and T).
// Returns false if A is singular in FP64.
#ifndef DQ_KAPPA_FP32_JET_MAX
#define DQ_KAPPA_FP32_JET_MAX 1.0e5f
#endif
__device__ __forceinline__ bool det_factor_jets(const float* A, float* LU, float* X0, float* R, float* T,
                                                float* Xhi, float* Xlo, double* LUd, double* Ainvd,
                                                const float* rmax, int* perm, int n, int lane,
                                                unsigned long long* n_fp64, int* sign, double* logabs) {
  const int nsq = n * n;
  bool fp64 = !warp_lu<float>(LU, perm, n, lane, sign, logabs);
  if (!fp64) {
    warp_inverse<float>(LU, perm, n, lane, X0);
    float imax = 0;
    for (int q = lane; q < nsq; q += 32) imax = fmaxf(imax, fabsf(X0[q]) * rmax[q - (q / n) * n]);
    const float kappa = float(n) * warp_max(imax);
    fp64 = !(kappa <= DQ_KAPPA_FP32_JET_MAX);
  }
  if (!fp64) {
    for (int q = lane; q < nsq; q += 32) {
      Xhi[q] = X0[q];
      Xlo[q] = 0.f;
    }
    __syncwarp();
    fp64 = true;  // until the residual has converged
    for (int it = 0; it < 4; ++it) {
      // residual R = I - A X
      float rm = 0.f;
      for (int q = lane; q < nsq; q += 32) {
        const int a = q / n, m = q - (q / n) * n;
        dfloat acc = {a == m ? -1.f : 0.f, 0.f};
        for (int l = 0; l < n; ++l) acc = dot2_step(acc, A[a * n + l], Xhi[l * n + m]);
        if (it > 0)
          for (int l = 0; l < n; ++l) acc = dot2_step(acc, A[a * n + l], Xlo[l * n + m]);
        R[q] = -(acc.hi + acc.lo);
        rm = fmaxf(rm, fabsf(acc.hi));
      }
      rm = warp_max(rm);
      if (!(rm <= 0.25f)) break;  // not contracting
      __syncwarp();
      // T = Xhi R, then X += T (the step squares the residual)
      for (int q = lane; q < nsq; q += 32) {
        const int a = q / n, m = q - (q / n) * n;
        float c = 0.f;
        for (int l = 0; l < n; ++l) c = fmaf(Xhi[a * n + l], R[l * n + m], c);
        T[q] = c;
      }
      __syncwarp();
      for (int q = lane; q < nsq; q += 32) {
        const dfloat x = two_sum(Xhi[q], T[q]);
        const dfloat y = quick_two_sum(x.hi, __fadd_rn(x.lo, Xlo[q]));
        Xhi[q] = y.hi;
        Xlo[q] = y.lo;
      }
      __syncwarp();
      if (rm <= 1e-4f) {  // X now accurate to about rm^2 <= 1e-8 relative
        fp64 = false;
        break;
      }
    }
  }
  if (!fp64) {
    // R = P A - L U (row r of P A is row perm[r] of A), then T = E = X P^T R:
    // E[a][c] = sum_r X[a][perm[r]] R[r][c]
    for (int q = lane; q < nsq; q += 32) {
      const int r = q / n, c = q - (q / n) * n;
      const int mm = r < c ? r : c;
      dfloat acc = {-A[perm[r] * n + c], 0.f};
      for (int m = 0; m <= mm; ++m) acc = dot2_step(acc, m == r ? 1.f : LU[r * n + m], LU[m * n + c]);
      R[q] = -(acc.hi + acc.lo);
    }
    __syncwarp();
    for (int q = lane; q < nsq; q += 32) {
      const int a = q / n, c = q - (q / n) * n;
      float e = 0.f;
      for (int r = 0; r < n; ++r) e = fmaf(Xhi[a * n + perm[r]], R[r * n + c], e);
      T[q] = e;
    }
    __syncwarp();
    float part = 0.f;
    for (int q = lane; q < nsq; q += 32) {
      const int a = q / n, c = q - (q / n) * n;
      part += (a == c ? T[q] : 0.f) + 0.5f * T[q] * T[c * n + a];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    *logabs += (double)part;
  } else {
    __syncwarp();
    if (lane == 0) atomicAdd(n_fp64, 1ull);
    for (int q = lane; q < nsq; q += 32) LUd[q] = (double)A[q];
    __syncwarp();
    if (!warp_lu<double>(LUd, perm, n, lane, sign, logabs)) return false;
    warp_inverse<double>(LUd, perm, n, lane, Ainvd);
    for (int q = lane; q < nsq; q += 32) {
      const double a = Ainvd[q];
      const float h = (float)a;
      Xhi[q] = h;
      Xlo[q] = (float)(a - (double)h);
    }
  }
  __syncwarp();
  return true;
}
constexpr int kDetNR = 8;

__host__ __device__ inline size_t det_jets_smem_per_warp(int nmax, int N3) {
  const size_t nn = (size_t)nmax * nmax;
  const size_t fl = nn * (14 + 4) + (size_t)(N3 + 1) * nmax * 2;  // float arrays
  const size_t bytes = fl * 4 + 2 * nn * 8 + 32 * 4;
  return (bytes + 15) / 16 * 16;
}

__device__ __forceinline__ void orbital_det_jets_kernel_body(const int64_t bx_, const int by_, const int64_t nbx_, const float* __restrict__ phi, const float* __restrict__ geo,
                            const float* __restrict__ params, int64_t Bc, int N, int n_up, int M, int K, int C,
                            int Wo, int E, int n_ee, int64_t om_up, int64_t om_dn, int64_t ze_up, int64_t ze_dn,
                            double* __restrict__ det, unsigned long long* __restrict__ n_fp64, int full) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int warps = blockDim.x / 32;
  const int64_t gw = (int64_t)bx_ * warps + warp;
  const int n_dn = N - n_up;
  const int nmax = full ? N : (n_up > n_dn ? n_up : n_dn);
  const int N3 = 3 * N;
  const int nn = nmax * nmax;
  unsigned char* base = smem_raw + warp * det_jets_smem_per_warp(nmax, N3);
  double* LUd = reinterpret_cast<double*>(base);  // FP64 fallback
  double* Ainvd = LUd + nn;
  float* A = reinterpret_cast<float*>(Ainvd + nn);
  float* LU = A + nn;
  float* X0 = LU + nn;
  float* Xhi = X0 + nn;
  float* Xlo = Xhi + nn;
  float* tmp = Xlo + nn;
  float* Th = tmp + nn;   // [2][nn] double-buffered X_t, high part
  float* Tl = Th + 2 * nn;  // [2][nn] low part
  float* env = Tl + 2 * nn;
  float* jenv = env + nn;  // [3][nn]
  float* lenv = jenv + 3 * nn;
  float* phi0 = lenv + nn;
  float* rmax = phi0 + nn;   // [nmax] row maxima of A (nn reserved)
  float* DG = rmax + nn;     // [N3 + 1][nmax][2] diagonals of X_t
  int* perm = reinterpret_cast<int*>(DG + (N3 + 1) * nmax * 2);

  if (gw >= Bc * 2 * K) return;
  const int64_t b = gw / (2 * K);
  const int s = (int)((gw / K) % 2);
  const int p = (int)(gw % K);
  int n, i0;
  det_block(s, N, n_up, full, n, i0);
  double* out = det + gw * (N3 + 3);
  if (n == 0) {  // empty determinant = 1
    for (int k = lane; k < N3 + 3; k += 32) out[k] = k == 0 ? 1.0 : 0.0;
    return;
  }
  const float* phib = phi + b * N * C * Wo;
  const float* gb = geo + b * E * 4;
  const int nsq = n * n;

  // Envelopes (Eq. 20) with their derivatives in the coordinates of electron i.
  for (int q = lane; q < nsq; q += 32) {
    const int ii = q / n, k = q - (q / n) * n, o = p * n + k, i = i0 + ii;
    const bool up = i < n_up;
    const float* om = params + (up ? om_up : om_dn);
    const float* ze = params + (up ? ze_up : ze_dn);
    float ev = 0, j0 = 0, j1 = 0, j2 = 0, lv = 0;
    for (int I = 0; I < M; ++I) {
      const float* g = gb + (n_ee + i * M + I) * 4;
      const float z = ze[o * M + I];
      const float w = om[o * M + I] * expf(-z * g[0]);
      ev += w;
      j0 -= w * z * g[1];
      j1 -= w * z * g[2];
      j2 -= w * z * g[3];
      lv += w * (z * z - 2.f * z / g[0]);
    }
    env[q] = ev;
    jenv[q] = j0;
    jenv[nn + q] = j1;
    jenv[2 * nn + q] = j2;
    lenv[q] = lv;
    const float f0 = phib[(int64_t)i * C * Wo + o];
    phi0[q] = f0;
    A[q] = f0 * ev;
    LU[q] = f0 * ev;
  }
  __syncwarp();
  if (lane < n) {
    float m = 0;
    for (int k = 0; k < n; ++k) m = fmaxf(m, fabsf(A[lane * n + k]));
    rmax[lane] = m;
  }
  __syncwarp();

  int sign = 0;
  double logabs = -INFINITY;
  if (!det_factor_jets(A, LU, X0, tmp, Th, Xhi, Xlo, LUd, Ainvd, rmax, perm, n, lane, n_fp64, &sign, &logabs)) {
    for (int k = lane; k < N3 + 3; k += 32) out[k] = k == 1 ? -INFINITY : 0.0;
    return;
  }
  if (lane == 0) {
    out[0] = (double)sign;
    out[1] = logabs;
  }

  // ---- tangents ----
  // entries owned by this lane: q = lane and lane + 32 (n <= kDetNR)
  int qa[2], ra[2], ma[2];
  float ah[2][kDetNR], al[2][kDetNR];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int q = lane + 32 * r;
    qa[r] = q < nsq ? q : -1;
    ra[r] = q < nsq ? q / n : 0;
    ma[r] = q < nsq ? q - (q / n) * n : 0;
#pragma unroll
    for (int l = 0; l < kDetNR; ++l) {
      ah[r][l] = l < n && q < nsq ? Xhi[ra[r] * n + l] : 0.f;
      al[r][l] = l < n && q < nsq ? Xlo[ra[r] * n + l] : 0.f;
    }
  }
  dfloat s2 = {0.f, 0.f};
  // the lane's entries of d_t A read one tangent ahead (the load of t + 1 overlaps the products
  // of t); the derivatives in the row's own electron are kept for the Laplacian
  const float* phq[2];
  float pre[2], dself[2][3];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    phq[r] = phib + (int64_t)(i0 + ra[r]) * C * Wo + p * n + ma[r];
    pre[r] = qa[r] >= 0 ? phq[r][(int64_t)1 * Wo] : 0.f;
    dself[r][0] = dself[r][1] = dself[r][2] = 0.f;
  }
  for (int t = 0; t <= N3; ++t) {
    const bool is_lap = t == N3;
    const int te = t / 3, tx = t - (t / 3) * 3;
    float cur[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      cur[r] = pre[r];
      if (qa[r] >= 0 && t < N3) pre[r] = phq[r][(int64_t)(t + 1 == N3 ? C - 1 : 2 + t) * Wo];
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (qa[r] < 0) continue;
      const int q = qa[r], i = i0 + ra[r];
      float v = cur[r] * env[q];
      if (is_lap) {
        v += phi0[q] * lenv[q];
#pragma unroll
        for (int x = 0; x < 3; ++x) v += 2.f * dself[r][x] * jenv[x * nn + q];
      } else if (te == i) {
        v += phi0[q] * jenv[tx * nn + q];
        dself[r][0] = tx == 0 ? cur[r] : dself[r][0];
        dself[r][1] = tx == 1 ? cur[r] : dself[r][1];
        dself[r][2] = tx == 2 ? cur[r] : dself[r][2];
      }
      tmp[q] = v;
    }
    __syncwarp();
    float* th = Th + (t & 1) * nn;
    float* tl = Tl + (t & 1) * nn;
    dfloat xv[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      xv[r] = {0.f, 0.f};
      if (qa[r] < 0) continue;
      const int m = ma[r];
      dfloat acc = {0.f, 0.f};
      float cl = 0.f;
#pragma unroll
      for (int l = 0; l < kDetNR; ++l) {
        if (l < n) {
          const float y = tmp[l * n + m];
          acc = dot2_step(acc, ah[r][l], y);
          cl = fmaf(al[r][l], y, cl);
        }
      }
      const dfloat x = quick_two_sum(acc.hi, __fadd_rn(acc.lo, cl));
      xv[r] = x;
      if (ra[r] == m) {
        DG[(t * nmax + m) * 2] = x.hi;
        DG[(t * nmax + m) * 2 + 1] = x.lo;
      }
      if (!is_lap) {
        th[qa[r]] = x.hi;
        tl[qa[r]] = x.lo;
      }
    }
    __syncwarp();
    if (!is_lap) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (qa[r] < 0) continue;
        const int tq = ma[r] * n + ra[r];  // transposed entry
        s2 = df_add(s2, df_mul(xv[r], {th[tq], tl[tq]}));
      }
    }
  }
  const dfloat s2s = warp_sum_df(s2);
  __syncwarp();
  for (int t = lane; t <= N3; t += 32) {
    dfloat tr = {0.f, 0.f};
    for (int a = 0; a < n; ++a) tr = df_add(tr, {DG[(t * nmax + a) * 2], DG[(t * nmax + a) * 2 + 1]});
    const double v = (double)tr.hi + (double)tr.lo;
    if (t < N3) out[2 + t] = v;
    else out[2 + N3] = v - ((double)s2s.hi + (double)s2s.lo);
  }
}

// ---------------------------------------------------------------------------
// Determinant jets of the FP32 modes for spin blocks of 9 to kDetNRL electrons:
// the factorisation of the small-block body (det_factor_jets), with a layout of
// the 3N + 1 tangent products X_t = A^-1 d_t A for larger blocks.  The warp's
// lanes form G = 32 / n column groups; lane (g, a) keeps row a of Xhi / Xlo in
// registers, forms the entries (a, k) of d_t A for the columns k of group g and
// computes X_t[a][k] for the same columns as compensated dot products whose
// second operand (column k of d_t A) is a shared-memory broadcast.  The Jacobian
// traces go through an 8-slot ring of per-row diagonals, summed once per 8
// tangents; sum_t tr(X_t^2) pairs each owned entry with its transpose.
// ---------------------------------------------------------------------------
constexpr int kDetNRL = 32;

__host__ __device__ inline size_t det_jets_large_smem_per_warp(int nmax) {
  const size_t nn = (size_t)nmax * nmax;
  const size_t bytes = (15 * nn + 17 * (size_t)nmax) * 4 + (size_t)nmax * 4;
  return (bytes + 15) / 16 * 16;
}

// Column-chunk width of the tangent products for an n x n block (3 to 8).
__host__ __device__ inline int det_large_cw(int n) {
  if (n <= 16) {
    const int G = 32 / n;
    return (n + G - 1) / G;
  }
  const int nch = (n + 7) / 8;
  return (n + nch - 1) / nch;
}

template <int NR, int CW>
__device__ __forceinline__ void det_tangents_large(const float* __restrict__ phr, const float* env,
                                                   const float* jenv, const float* lenv, const float* phi0,
                                                   const float* xh, const float* xl, float* tmp, float* Th,
                                                   float* Tl, float* DG, int n, int nn, int nmax, int i, int a,
                                                   int cb, int ce, bool active, int C, int Wo, int N3, int lane,
                                                   double* out) {
  dfloat s2 = {0.f, 0.f};
  float lap_tr = 0.f, lap_lo = 0.f;
  // blocks of at most 16 (one column chunk per lane): the lane's entries of d_t A are read one
  // tangent ahead, so that the loads of t + 1 overlap the products of t
  constexpr bool kAhead = NR <= 16;
  float pre[CW];
#pragma unroll
  for (int j = 0; j < CW; ++j) pre[j] = kAhead && cb + j < ce ? phr[(int64_t)1 * Wo + cb + j] : 0.f;
  for (int t = 0; t <= N3; ++t) {
    const bool is_lap = t == N3;
    const int c = is_lap ? C - 1 : 1 + t;
    const int te = t / 3, tx = t - (t / 3) * 3;
    float* dA = tmp + (t & 1) * nn;
    float cur[CW];
#pragma unroll
    for (int j = 0; j < CW; ++j) {
      cur[j] = pre[j];
      if (kAhead && t < N3 && cb + j < ce) pre[j] = phr[(int64_t)(t + 1 == N3 ? C - 1 : 2 + t) * Wo + cb + j];
    }
    for (int k0 = cb; k0 < ce; k0 += CW) {
#pragma unroll
      for (int j = 0; j < CW; ++j) {
        const int k = k0 + j;
        if (k < ce) {
          const int q = a * n + k;
          float v = (kAhead ? cur[j] : phr[(int64_t)c * Wo + k]) * env[q];
          if (is_lap) {
            v += phi0[q] * lenv[q];
            for (int x = 0; x < 3; ++x) v += 2.f * phr[(int64_t)(1 + 3 * i + x) * Wo + k] * jenv[x * nn + q];
          } else if (te == i) {
            v += phi0[q] * jenv[tx * nn + q];
          }
          dA[q] = v;
        }
      }
    }
    __syncwarp();
    float* th = Th + (t & 1) * nn;
    float* tl = Tl + (t & 1) * nn;
    for (int c0 = cb; c0 < ce; c0 += CW) {
      dfloat acc[CW];
      float cl[CW];
#pragma unroll
      for (int j = 0; j < CW; ++j) {
        acc[j] = {0.f, 0.f};
        cl[j] = 0.f;
      }
      // columns c0 .. c0 + CW - 1 of d_t A; those past ce (at most the next
      // row's first entries, inside the warp's buffers) are computed and dropped
#pragma unroll
      for (int l = 0; l < NR; ++l) {
        if (l >= n) break;
        const float* yr = dA + l * n + c0;
#pragma unroll
        for (int j = 0; j < CW; ++j) {
          const float y = yr[j];
          acc[j] = dot2_step(acc[j], xh[l], y);
          cl[j] = fmaf(xl[l], y, cl[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < CW; ++j) {
        const int m = c0 + j;
        if (m < ce) {
          const dfloat x = quick_two_sum(acc[j].hi, __fadd_rn(acc[j].lo, cl[j]));
          if (m == a) {
            DG[((t & 7) * nmax + a) * 2] = x.hi;
            DG[((t & 7) * nmax + a) * 2 + 1] = x.lo;
          }
          if (!is_lap) {
            th[a * n + m] = x.hi;
            tl[a * n + m] = x.lo;
          }
        }
      }
    }
    __syncwarp();
    if (!is_lap && active) {
      for (int m = cb; m < ce; ++m)
        s2 = df_add(s2, df_mul({th[a * n + m], tl[a * n + m]}, {th[m * n + a], tl[m * n + a]}));
    }
    if ((t & 7) == 7 || is_lap) {
      // traces of the last (t & 7) + 1 tangents: lane j sums slot j over the rows
      const int t0 = t - (t & 7);
      if (lane <= (t & 7)) {
        dfloat tr = {0.f, 0.f};
        for (int r = 0; r < n; ++r) tr = df_add(tr, {DG[(lane * nmax + r) * 2], DG[(lane * nmax + r) * 2 + 1]});
        if (t0 + lane < N3) {
          out[2 + t0 + lane] = (double)tr.hi + (double)tr.lo;
        } else {
          lap_tr = tr.hi;
          lap_lo = tr.lo;
        }
      }
      __syncwarp();
    }
  }
  const dfloat s2s = warp_sum_df(s2);
  if (lane == (N3 & 7)) out[2 + N3] = ((double)lap_tr + (double)lap_lo) - ((double)s2s.hi + (double)s2s.lo);
}

template <int NR>
__device__ __forceinline__ void orbital_det_jets_large_body(const int64_t bx_, const int64_t nbx_, const float* __restrict__ phi,
                            const float* __restrict__ geo, const float* __restrict__ params, int64_t Bc, int N,
                            int n_up, int M, int K, int C, int Wo, int E, int n_ee, int64_t om_up, int64_t om_dn,
                            int64_t ze_up, int64_t ze_dn, double* __restrict__ det,
                            unsigned long long* __restrict__ n_fp64, int full) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int warps = blockDim.x / 32;
  const int64_t gw = (int64_t)bx_ * warps + warp;
  const int n_dn = N - n_up;
  const int nmax = full ? N : (n_up > n_dn ? n_up : n_dn);
  const int N3 = 3 * N;
  const int nn = nmax * nmax;
  unsigned char* base = smem_raw + warp * det_jets_large_smem_per_warp(nmax);
  // persistent: envelope jets and phi values of the block
  float* env = reinterpret_cast<float*>(base);
  float* jenv = env + nn;  // [3][nn]
  float* lenv = jenv + 3 * nn;
  float* phi0 = lenv + nn;
  // factorisation (9 nn floats); the tangent buffers tmp[2], Th[2], Tl[2] reuse
  // the first 6 nn of it once Xhi / Xlo are in registers
  float* W = phi0 + nn;
  double* LUd = reinterpret_cast<double*>(W);
  double* Ainvd = LUd + nn;
  float* A = W + 4 * nn;
  float* LU = A + nn;
  float* X0 = LU + nn;
  float* Xhi = X0 + nn;
  float* Xlo = Xhi + nn;
  float* tmp = W;
  float* Th = W + 2 * nn;
  float* Tl = W + 4 * nn;
  float* DG = W + 9 * nn;  // [8][nmax][2]
  float* rmax = DG + 16 * nmax;
  int* perm = reinterpret_cast<int*>(rmax + nmax);

  if (gw >= Bc * 2 * K) return;
  const int64_t b = gw / (2 * K);
  const int s = (int)((gw / K) % 2);
  const int p = (int)(gw % K);
  int n, i0;
  det_block(s, N, n_up, full, n, i0);
  double* out = det + gw * (N3 + 3);
  if (n == 0) {  // empty determinant = 1
    for (int k = lane; k < N3 + 3; k += 32) out[k] = k == 0 ? 1.0 : 0.0;
    return;
  }
  const float* phib = phi + b * N * C * Wo;
  const float* gb = geo + b * E * 4;
  const int nsq = n * n;

  // Envelopes (Eq. 20) with their derivatives in the coordinates of electron i
  // (block-local row stride n).
  for (int q = lane; q < nsq; q += 32) {
    const int ii = q / n, k = q - (q / n) * n, o = p * n + k, i = i0 + ii;
    const bool up = i < n_up;
    const float* om = params + (up ? om_up : om_dn);
    const float* ze = params + (up ? ze_up : ze_dn);
    float ev = 0, j0 = 0, j1 = 0, j2 = 0, lv = 0;
    for (int I = 0; I < M; ++I) {
      const float* g = gb + (n_ee + i * M + I) * 4;
      const float z = ze[o * M + I];
      const float w = om[o * M + I] * expf(-z * g[0]);
      ev += w;
      j0 -= w * z * g[1];
      j1 -= w * z * g[2];
      j2 -= w * z * g[3];
      lv += w * (z * z - 2.f * z / g[0]);
    }
    env[q] = ev;
    jenv[q] = j0;
    jenv[nn + q] = j1;
    jenv[2 * nn + q] = j2;
    lenv[q] = lv;
    const float f0 = phib[(int64_t)i * C * Wo + o];
    phi0[q] = f0;
    A[q] = f0 * ev;
    LU[q] = f0 * ev;
  }
  __syncwarp();
  if (lane < n) {
    float m = 0;
    for (int k = 0; k < n; ++k) m = fmaxf(m, fabsf(A[lane * n + k]));
    rmax[lane] = m;
  }
  __syncwarp();

  int sign = 0;
  double logabs = -INFINITY;
  // R, T = W[0, 2 nn): the LUd area, used only on the other branch
  if (!det_factor_jets(A, LU, X0, W, W + nn, Xhi, Xlo, LUd, Ainvd, rmax, perm, n, lane, n_fp64, &sign, &logabs)) {
    for (int k = lane; k < N3 + 3; k += 32) out[k] = k == 1 ? -INFINITY : 0.0;
    return;
  }
  if (lane == 0) {
    out[0] = (double)sign;
    out[1] = logabs;
  }

  const int G = n <= 16 ? 32 / n : 1;
  const int g = lane / n, a = lane - (lane / n) * n;
  const bool active = g < G;
  const int cw = (n + G - 1) / G;
  const int cb = active ? g * cw : 0;
  const int ce = active ? min(n, cb + cw) : 0;
  float xh[NR], xl[NR];
#pragma unroll
  for (int l = 0; l < NR; ++l) {
    xh[l] = active && l < n ? Xhi[a * n + l] : 0.f;
    xl[l] = active && l < n ? Xlo[a * n + l] : 0.f;
  }
  __syncwarp();  // A, LU and the FP64 area become the tangent buffers
  const int i = i0 + (active ? a : 0);
  const float* phr = phib + (int64_t)i * C * Wo + p * n;
  switch (det_large_cw(n)) {
    case 3:
    case 4:
      det_tangents_large<NR, 4>(phr, env, jenv, lenv, phi0, xh, xl, tmp, Th, Tl, DG, n, nn, nmax, i, a, cb, ce,
                                active, C, Wo, N3, lane, out);
      break;
    case 5:
    case 6:
      det_tangents_large<NR, 6>(phr, env, jenv, lenv, phi0, xh, xl, tmp, Th, Tl, DG, n, nn, nmax, i, a, cb, ce,
                                active, C, Wo, N3, lane, out);
      break;
    case 7:
      det_tangents_large<NR, 7>(phr, env, jenv, lenv, phi0, xh, xl, tmp, Th, Tl, DG, n, nn, nmax, i, a, cb, ce,
                                active, C, Wo, N3, lane, out);
      break;
    default:
      det_tangents_large<NR, 8>(phr, env, jenv, lenv, phi0, xh, xl, tmp, Th, Tl, DG, n, nn, nmax, i, a, cb, ce,
                                active, C, Wo, N3, lane, out);
      break;
  }
}

// The large-block jet body over several molecules, NR = 16 (tag 2) or kDetNRL
// (tag 3); a kernel of its own so that its registers do not lower the occupancy
// of the small-block body.
template <int NR>
__global__ void __launch_bounds__(128) orbital_det_large_group(const __grid_constant__ Grp<orbital_det_kernel_args<float>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  const orbital_det_kernel_args<float>& a_ = g.a[m_];
  orbital_det_jets_large_body<NR>(l_, g.nbx[m_], a_.phi, a_.geo, a_.params, a_.Bc, a_.N, a_.n_up, a_.M, a_.K, a_.C,
                                  a_.Wo, a_.E, a_.n_ee, a_.om_up, a_.om_dn, a_.ze_up, a_.ze_dn, a_.det, a_.n_fp64,
                                  a_.full);
}

// Determinants of several molecules in one launch (FP32 modes): tag 1 runs the
// FP32 jet kernel body (spin blocks of at most kDetNR electrons), tag 0 the
// general body (value-only calls, blocks too large for the jet bodies).  Both
// use four warps per CTA, one matrix per warp.
__global__ void __launch_bounds__(128) orbital_det_mixed_group(const __grid_constant__ Grp<orbital_det_kernel_args<float>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  const orbital_det_kernel_args<float>& a_ = g.a[m_];
  const int tag = g.tag[m_];
  if (tag == 1)
    orbital_det_jets_kernel_body(l_, 0, g.nbx[m_], a_.phi, a_.geo, a_.params, a_.Bc, a_.N, a_.n_up, a_.M, a_.K, a_.C,
                                 a_.Wo, a_.E, a_.n_ee, a_.om_up, a_.om_dn, a_.ze_up, a_.ze_dn, a_.det, a_.n_fp64,
                                 a_.full);
  else
    orbital_det_kernel_body<float>(l_, 0, g.nbx[m_], a_.phi, a_.geo, a_.params, a_.Bc, a_.N, a_.n_up, a_.M, a_.K,
                                   a_.C, a_.Wo, a_.E, a_.n_ee, a_.om_up, a_.om_dn, a_.ze_up, a_.ze_dn, a_.det,
                                   a_.n_fp64, a_.full);
}

// Sum of embeddings over electrons, the input of the Jastrow factor (Eq. 24).
template <class T>
struct jastrow_sum_kernel_args {
  const T* F;
  int64_t Bc;
  int N;
  int C;
  int D;
  T* js;
};

template <class T>
__device__ __forceinline__ void jastrow_sum_kernel_body(const int64_t bx_, const int by_, const int64_t nbx_, const T* __restrict__ F, int64_t Bc, int N, int C, int D, T* __restrict__ js) {
  const int64_t gid = (int64_t)bx_ * blockDim.x + threadIdx.x;
  if (gid >= Bc * C * D) return;
  const int64_t b = gid / (C * D);
  const int64_t cd = gid % (C * D);
  T acc = 0;
  for (int i = 0; i < N; ++i) acc += F[(b * N + i) * C * D + cd];
  js[gid] = acc;
}

// One launch over several molecules: block b runs entry m of the table.
template <class T>
__global__ void jastrow_sum_kernel_group(const __grid_constant__ Grp<jastrow_sum_kernel_args<T>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  GRP_STATIC(m_, const auto& a_ = g.a[K_];
             jastrow_sum_kernel_body<T>(grp_bx(g, K_, l_), grp_by(g, K_, l_), g.nbx[K_], a_.F, a_.Bc, a_.N, a_.C, a_.D, a_.js);)
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
struct combine_kernel_args {
  const double* det;
  const T* jh;
  const T* geo;
  const T* params;
  const double* Zn;
  const int* pair_ij;
  const int* pair_of;
  int64_t Bc;
  int N;
  int n_up;
  int M;
  int K;
  int C;
  int D;
  int E;
  int n_ee;
  int64_t c_off;
  int64_t wJ2_off;
  int use_jastrow;
  int use_cusp;
  double alpha;
  double Vnn;
  T* logabs;
  int8_t* sign_out;
  T* e_loc;
  T* grad_out;
  unsigned int* status;
};

template <class T>
__device__ __forceinline__ void combine_kernel_body(const int64_t bx_, const int by_, const int64_t nbx_, const double* __restrict__ det, const T* __restrict__ jh, const T* __restrict__ geo,
                   const T* __restrict__ params, const double* __restrict__ Zn, const int* __restrict__ pair_ij,
                   const int* __restrict__ pair_of, int64_t Bc, int N, int n_up, int M, int K, int C, int D, int E, int n_ee, int64_t c_off,
                   int64_t wJ2_off, int use_jastrow, int use_cusp, double alpha, double Vnn, T* __restrict__ logabs,
                   int8_t* __restrict__ sign_out, T* __restrict__ e_loc, T* __restrict__ grad_out,
                   unsigned int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N3 = 3 * N;
  double* wp = reinterpret_cast<double*>(smem_raw);  // [K] determinant weights
  double* gsq = wp + K;                              // [K] |grad l_p|^2
  double* td = gsq + K;                              // [3][D] Jastrow: w t, w t', w t''
  double* red = td + 3 * D;                          // [32]
  double* gJk = red + 32;                            // [3N] Jastrow gradient components
  __shared__ double s_scalar[4];
  const int64_t b = bx_;
  const int tid = threadIdx.x;
  const bool jets = C > 1;
  const double* db = det + b * 2 * K * (N3 + 3);
  auto dp = [&](int s, int p) { return db + ((int64_t)s * K + p) * (N3 + 3); };

  // log-sum-exp over determinant pairs (Eq. 28), warp 0 with lanes over pairs
  if (tid < 32) {
    double lmax = -INFINITY;
    for (int p = tid; p < K; p += 32) {
      const double cp = (double)params[c_off + p];
      const double sp = dp(0, p)[0] * dp(1, p)[0] * (cp > 0 ? 1.0 : cp < 0 ? -1.0 : 0.0);
      const double lp = sp != 0.0 ? dp(0, p)[1] + dp(1, p)[1] + log(fabs(cp)) : -INFINITY;
      wp[p] = lp;
      gsq[p] = sp;
      if (sp != 0.0 && lp > lmax) lmax = lp;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    double S = 0.0;  // summed in a fixed order below: per lane, then a butterfly
    if (lmax > -INFINITY)
      for (int p = tid; p < K; p += 32) {
        const double e = gsq[p] != 0.0 ? gsq[p] * exp(wp[p] - lmax) : 0.0;
        wp[p] = e;
        S += e;
      }
    else
      for (int p = tid; p < K; p += 32) wp[p] = 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
    for (int p = tid; p < K; p += 32) wp[p] = S != 0.0 ? wp[p] / S : 0.0;
    if (tid == 0) {
      s_scalar[0] = S > 0 ? 1.0 : (S < 0 ? -1.0 : 0.0);
      s_scalar[1] = S != 0.0 ? lmax + log(fabs(S)) : -INFINITY;
    }
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
  // Jastrow gradient components and Laplacian term: one warp per coordinate k, lanes over
  // features (coalesced rows of the Jastrow-input jets)
  double lJpart = 0.0;
  if (use_jastrow) {
    const int wq = tid / 32, ln = tid % 32;
    for (int k = wq; k < N3; k += kCombineThreads / 32) {
      const T* row = jb + (int64_t)(1 + k) * D;
      double gj = 0.0, lj = 0.0;
      for (int a = ln; a < D; a += 32) {
        const double h = (double)row[a];
        gj += td[D + a] * h;
        lj += td[2 * D + a] * h * h;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        gj += __shfl_xor_sync(0xffffffffu, gj, o);
        lj += __shfl_xor_sync(0xffffffffu, lj, o);
      }
      if (ln == 0) {
        gJk[k] = gj;
        lJpart += lj;
      }
    }
    __syncthreads();
  }
  // gradient components
  double g2part = 0.0;
  for (int k = tid; k < N3; k += kCombineThreads) {
    double g = 0.0;
    for (int p = 0; p < K; ++p) g += wp[p] * (dp(0, p)[2 + k] + dp(1, p)[2 + k]);
    if (use_jastrow) g += gJk[k];
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
    if (grad_out) grad_out[b * N3 + k] = (T)g;  // d log|psi| / d r_k
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

// One launch over several molecules: block b runs entry m of the table.
template <class T>
__global__ void __launch_bounds__(kCombineThreads) combine_kernel_group(const __grid_constant__ Grp<combine_kernel_args<T>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  GRP_STATIC(m_, const auto& a_ = g.a[K_];
             combine_kernel_body<T>(grp_bx(g, K_, l_), grp_by(g, K_, l_), g.nbx[K_], a_.det, a_.jh, a_.geo, a_.params, a_.Zn, a_.pair_ij, a_.pair_of, a_.Bc, a_.N, a_.n_up, a_.M, a_.K, a_.C, a_.D, a_.E, a_.n_ee, a_.c_off, a_.wJ2_off, a_.use_jastrow, a_.use_cusp, a_.alpha, a_.Vnn, a_.logabs, a_.sign_out, a_.e_loc, a_.grad_out, a_.status);)
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Single-molecule launchers: the grouped kernels with a one-entry table, so that
// a molecule gives the same bits alone and in a batch.
template <class T>
cudaError_t launch_geometry(const dq_handle_s& h, const FwdDims& d, const T* r, FwdBuffers<T> b, cudaStream_t s) {
  const MolFwd<T> m{&h, d, nullptr, b};
  return launch_geometry_group<T>(&m, 1, &r, s);
}

template <class T>
cudaError_t launch_edge_hidden(const dq_handle_s& h, const FwdDims& d, const T* params, int l, FwdBuffers<T> b,
                               cudaStream_t s) {
  const MolFwd<T> m{&h, d, params, b};
  return launch_edge_hidden_group<T>(&m, 1, l, s);
}

template <class T>
cudaError_t launch_layer0_node(const dq_handle_s& h, const FwdDims& d, const T* params, FwdBuffers<T> b,
                               cudaStream_t s) {
  const MolFwd<T> m{&h, d, params, b};
  return launch_layer0_node_group<T>(&m, 1, s);
}

namespace {
template <class T>
constexpr int msg_ib() { return sizeof(T) == 4 ? 8 : 4; }
}  // namespace

template <class T>
cudaError_t launch_messages(const dq_handle_s& h, const FwdDims& d, const T* params, int l, bool z_const,
                            FwdBuffers<T> b, cudaStream_t s) {
  const MolFwd<T> m{&h, d, params, b};
  return launch_messages_group<T>(&m, 1, l, z_const, s);
}

template <class T>
cudaError_t launch_update(const dq_handle_s& h, const FwdDims& d, const T* params, bool from_spin, FwdBuffers<T> b,
                          cudaStream_t s) {
  const MolFwd<T> m{&h, d, params, b};
  return launch_update_group<T>(&m, 1, from_spin, s);
}

template <class T>
cudaError_t launch_update_io(const dq_handle_s& h, const FwdDims& d, const T* params, bool from_spin, const T* P,
                             const T* Fin, T* Fout, cudaStream_t s, void* Fbf) {
  update_kernel<T><<<blocks(d.Bc * d.N * d.D, 256), 256, 0, s>>>(P, Fin, Fout, params + std::max<int64_t>(h.off.E_spin, 0), d.Bc, d.N,
                                                                 d.n_up, d.C, d.D, from_spin ? 1 : 0,
                                                                 static_cast<__nv_bfloat16*>(Fbf));
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* src, void* dst, int64_t n, cudaStream_t s) {
  to_bf16_kernel<<<blocks(n, 256), 256, 0, s>>>(src, static_cast<__nv_bfloat16*>(dst), n);
  return cudaGetLastError();
}

// Which determinant body runs a molecule's matrices (the group kernel's tag) and
// its dynamic shared memory for four warps: 1 the small-block FP32 jet body,
// 2 / 3 the large-block FP32 jet body, 0 the general body.
template <class T>
int det_body_tag(int nmax, int N, int C, size_t* smem4) {
  const int nn = nmax * nmax;
  if (sizeof(T) == 4 && C > 1) {
    if (nmax <= kDetNR) {
      *smem4 = det_jets_smem_per_warp(nmax, 3 * N) * 4;
      return 1;
    }
    if (nmax <= kDetNRL && det_jets_large_smem_per_warp(nmax) * 4 <= 200 * 1024) {
      *smem4 = det_jets_large_smem_per_warp(nmax) * 4;
      return nmax <= 16 ? 2 : 3;
    }
  }
  *smem4 = ((size_t)nn * (3 * sizeof(double) + 10 * sizeof(T)) + 32 * sizeof(int) + 15) / 16 * 16 * 4;
  return 0;
}

template <class T>
cudaError_t launch_orbital_det(const dq_handle_s& h, const FwdDims& d, const T* params, FwdBuffers<T> b,
                               cudaStream_t s) {
  const int nmax = h.det_n();
  const int nn = nmax * nmax;
  {
    size_t sm4 = 0;
    const int tag = det_body_tag<T>(nmax, d.N, d.C, &sm4);
    if (tag != 0 || sm4 <= 200 * 1024) {
      const MolFwd<T> m{&h, d, params, b};
      return launch_orbital_det_group<T>(&m, 1, s);
    }
  }
  // spin blocks too large for four warps per CTA: one matrix per CTA
  const size_t per_warp = ((size_t)nn * (3 * sizeof(double) + 10 * sizeof(T)) + 32 * sizeof(int) + 15) / 16 * 16;
  const int warps = per_warp * 4 <= 200 * 1024 ? 4 : 1;
  const size_t smem = per_warp * warps;
  auto kern = orbital_det_kernel<T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t nmat = d.Bc * 2 * d.K;
  kern<<<blocks(nmat, warps), warps * 32, smem, s>>>(b.phi, b.geo, params, d.Bc, d.N, d.n_up, d.M, d.K, d.C,
                                                     d.K * nmax, h.edges.n_all, h.edges.n_ee, h.off.omega[0],
                                                     h.off.omega[1], h.off.zeta[0], h.off.zeta[1], b.det,
                                                     h.d_fp64_count, h.full_det);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_jastrow_sum(const dq_handle_s& h, const FwdDims& d, FwdBuffers<T> b, cudaStream_t s) {
  const MolFwd<T> m{&h, d, nullptr, b};
  return launch_jastrow_sum_group<T>(&m, 1, s);
}

template <class T>
cudaError_t launch_combine(const dq_handle_s& h, const FwdDims& d, const T* params, FwdBuffers<T> b, T* logabs,
                           int8_t* sign, T* e_loc, cudaStream_t s, T* grad) {
  const MolFwd<T> m{&h, d, params, b};
  return launch_combine_group<T>(&m, 1, &logabs, &sign, &e_loc, &grad, s);
}

// ---------------------------------------------------------------------------
// Grouped launches: one launch per step over every molecule of a batch, each
// molecule with its own dimensions, parameters and buffers (entry m of the
// launch's table).  Block counts per molecule are those of the single-molecule
// launchers above; dynamic shared memory is the largest any entry needs.
// ---------------------------------------------------------------------------
namespace {
int device_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}
template <class A>
cudaError_t check_group(const Grp<A>& g) {
  if (g.blocks() <= 0) return cudaSuccess;
  return g.blocks() > (int64_t)INT32_MAX ? cudaErrorInvalidConfiguration : cudaSuccess;
}
}  // namespace

template <class T>
cudaError_t launch_geometry_group(const MolFwd<T>* m, int n, const T* const* r, cudaStream_t s) {
  if (n > kMaxGroup) return cudaErrorInvalidValue;
  Grp<geometry_kernel_args<T>> g{};
  for (int k = 0; k < n; ++k) {
    const dq_handle_s& h = *m[k].h;
    const FwdDims& d = m[k].d;
    if (d.Bc <= 0) continue;
    const T* R = nullptr;
    if constexpr (sizeof(T) == 8) R = h.d_R; else R = h.d_Rf;
    g.add({r[k], R, h.d_pair_ij, d.Bc, d.N, d.M, h.edges.n_ee, h.edges.n_all, d.Q, d.C > 1 ? 3 : 1, h.rc, m[k].b.geo,
           m[k].b.rbf},
          blocks(d.Bc * h.edges.n_all, 128));
  }
  if (g.n == 0) return cudaSuccess;
  cudaError_t e = check_group(g);
  if (e != cudaSuccess) return e;
  geometry_kernel_group<T><<<(unsigned)g.blocks(), 128, 0, s>>>(g);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_edge_hidden_group(const MolFwd<T>* m, int n, int l, cudaStream_t s) {
  if (n > kMaxGroup) return cudaErrorInvalidValue;
  Grp<edge_hidden_kernel_args<T>> g{};
  size_t smem = 0;
  int64_t rows_all = 0;
  for (int k = 0; k < n; ++k) rows_all += m[k].d.Bc > 0 ? m[k].d.Bc * m[k].h->edges.n_all : 0;
  const int64_t grid_all = (int64_t)device_sms() * 6;  // persistent, 6 CTAs per SM, shared by row count
  for (int k = 0; k < n; ++k) {
    const dq_handle_s& h = *m[k].h;
    const FwdDims& d = m[k].d;
    if (d.Bc <= 0) continue;
    const int ej = d.C > 1 ? 3 : 1;
    const auto& y = h.off.layer[l];
    const int64_t rows = d.Bc * h.edges.n_all;
    smem = std::max(smem, ((size_t)3 * d.Q * d.D + 3 * d.D + (size_t)kEdgesPerCta * ej * d.Q) * sizeof(T));
    const int64_t nblk = (rows + kEdgesPerCta - 1) / kEdgesPerCta;
    int64_t share = (grid_all * rows + rows_all - 1) / rows_all;
    share = std::max<int64_t>(1, std::min(share, nblk));
    g.add({m[k].b.rbf, m[k].params, d.Bc, h.edges.n_all, h.edges.n_par, h.edges.n_ee, d.D, d.Q, ej, y.W1[0], y.W1[1],
           y.W1[2], y.b1[0], y.b1[1], y.b1[2], m[k].b.eh},
          share);
  }
  if (g.n == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(edge_hidden_kernel_group<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  edge_hidden_kernel_group<T><<<(unsigned)g.blocks(), kHiddenThreads, smem, s>>>(g);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_edge_update_group(const MolFwd<T>* m, int n, int l, const T* const* src, T* const* dst,
                                     cudaStream_t s) {
  if (n > kMaxGroup) return cudaErrorInvalidValue;
  Grp<edge_update_kernel_args<T>> g{};
  size_t smem = 0;
  for (int k = 0; k < n; ++k) {
    const dq_handle_s& h = *m[k].h;
    const FwdDims& d = m[k].d;
    if (d.Bc <= 0 || !h.edge_update || l < 1) continue;
    const int ej = d.C > 1 ? 3 : 1, Q = d.Q;
    const auto& y = h.off.layer[l];
    const int rpi = 256 / Q;
    const int64_t rows = d.Bc * h.edges.n_all, nblk = (rows + rpi - 1) / rpi;
    smem = std::max(smem, ((size_t)3 * Q * Q + 3 * Q + (size_t)rpi * ej * Q) * sizeof(T));
    g.add({src[k], dst[k], m[k].params, d.Bc, h.edges.n_all, h.edges.n_par, h.edges.n_ee, Q, ej, y.U[0], y.U[1],
           y.U[2], y.c[0], y.c[1], y.c[2]},
          std::max<int64_t>(1, std::min<int64_t>(nblk, (int64_t)device_sms() * 8)));
  }
  if (g.n == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(edge_update_kernel_group<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  e = check_group(g);
  if (e != cudaSuccess) return e;
  edge_update_kernel_group<T><<<(unsigned)g.blocks(), 256, smem, s>>>(g);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_el_init(const dq_handle_s& h, const FwdDims& d, const T* params, const T* r, T* F, void* Fbf, T* H0,
                           T* X0, cudaStream_t s) {
  if (d.Bc <= 0) return cudaSuccess;
  const int D = h.D, M3 = 3 * h.M, nch = d.C > 1 ? 5 : 1;
  int per = (int)std::min<size_t>(kElInitMax, (96 * 1024) / ((size_t)nch * D * sizeof(T) + M3 * sizeof(T)));
  per = std::max(per, 1);
  const size_t smem = (size_t)per * (M3 + nch * D) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(el_init_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const T* R = sizeof(T) == 8 ? reinterpret_cast<const T*>(h.d_R) : reinterpret_cast<const T*>(h.d_Rf);
  const int64_t n_el = d.Bc * h.N;
  el_init_kernel<T><<<(unsigned)((n_el + per - 1) / per), D, smem, s>>>(
      r, R, params, h.off.W_e1, h.off.b_e1, h.off.W_e2, h.off.b_e2, d.Bc, h.N, h.M, D, d.C, per, F,
      static_cast<__nv_bfloat16*>(Fbf), H0, X0);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_edge_update(const dq_handle_s& h, const FwdDims& d, const T* params, int l, const T* src, T* dst,
                               cudaStream_t s) {
  const MolFwd<T> m{&h, d, params, FwdBuffers<T>{}};
  return launch_edge_update_group<T>(&m, 1, l, &src, &dst, s);
}

template <class T>
cudaError_t launch_layer0_node_group(const MolFwd<T>* m, int n, cudaStream_t s) {
  if (n > kMaxGroup) return cudaErrorInvalidValue;
  Grp<layer0_node_kernel_args<T>> g{};
  for (int k = 0; k < n; ++k) {
    const dq_handle_s& h = *m[k].h;
    if (h.el_init) continue;  // no spin embeddings: layer 0 takes the general path
    g.add({m[k].params, m[k].d.D, h.off.E_spin, h.off.layer[0].W_h, m[k].b.z0}, blocks(2 * m[k].d.D, 128));
  }
  if (g.n == 0) return cudaSuccess;
  layer0_node_kernel_group<T><<<(unsigned)g.blocks(), 128, 0, s>>>(g);
  return cudaGetLastError();
}

namespace {
template <class T, class TO, int IB>
cudaError_t launch_messages_group_t(const MolFwd<T>* m, int n, int l, bool z_const, bool bf_out, cudaStream_t s) {
  auto out_of = [&](const MolFwd<T>& q) -> TO* {
    if constexpr (sizeof(TO) == 2) return static_cast<TO*>(q.b.msg_bf);
    else return reinterpret_cast<TO*>(q.b.msg);
  };
  (void)bf_out;
  if (m[0].d.C == 1) {
    Grp<messages_value_kernel_args<T, TO>> g{};
    size_t smem = 0;
    int threads = 32;
    for (int k = 0; k < n; ++k) threads = std::max(threads, 32 * (m[k].d.N < 8 ? m[k].d.N : 8));
    for (int k = 0; k < n; ++k) {
      const dq_handle_s& h = *m[k].h;
      const FwdDims& d = m[k].d;
      if (d.Bc <= 0) continue;
      smem = std::max(smem, (size_t)d.N * 32 * sizeof(T) + (size_t)d.N * d.N * sizeof(int));
      g.add({m[k].b.Z, m[k].b.z0, m[k].b.ew, m[k].params + h.off.layer[l].Y, h.d_pair_of, d.Bc, d.N, d.n_up, d.M, d.D,
             h.edges.n_all, h.edges.n_ee, z_const && !h.el_init ? 1 : 0, out_of(m[k])},
            d.Bc, (d.D + 31) / 32);
    }
    if (g.n == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(messages_value_kernel_group<T, TO>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = check_group(g);
    if (e != cudaSuccess) return e;
    messages_value_kernel_group<T, TO><<<(unsigned)g.blocks(), threads, smem, s>>>(g);
    return cudaGetLastError();
  }
  constexpr int CB = sizeof(T) == 4 ? 4 : 2;
  struct Ent {
    messages_kernel_args<T, TO> a;
    int64_t bx;
    int ny, L, smem, occ;
  };
  Ent ent[kMaxGroup];
  int ne = 0, smem = 0;
  for (int k = 0; k < n; ++k) {
    const dq_handle_s& h = *m[k].h;
    const FwdDims& d = m[k].d;
    if (d.Bc <= 0) continue;
    if (d.D % kMsgLanes) return cudaErrorInvalidConfiguration;
    if constexpr (sizeof(T) == 4) {
      // node channels from the node map: the sender-tiled kernel of messages_large.cu for the
      // molecules past the fused kernel's size (or when the handle asks for it)
      const bool tiled = h.msg_kernel == 2 || (h.msg_kernel == 0 && d.N > 16);
      if (tiled && !(z_const && !h.el_init) && messages_large_supported(h, d)) {
        cudaError_t e = launch_messages_large(h, d, reinterpret_cast<const float*>(m[k].params), l,
                                              reinterpret_cast<const float*>(m[k].b.Z),
                                              reinterpret_cast<const float*>(m[k].b.ew),
                                              reinterpret_cast<const float*>(m[k].b.geo), out_of(m[k]),
                                              sizeof(TO) == 2, s);
        if (e != cudaSuccess) return e;
        continue;
      }
    }
    bool stage_w1 = true;
    int L = kMsgLanes;
    MsgSmem lay = msg_smem_layout<T>(d.N, IB, CB, stage_w1, L);
    if (lay.total_bytes > 112 * 1024) {
      stage_w1 = false;
      lay = msg_smem_layout<T>(d.N, IB, CB, stage_w1, L);
      // 16 features per CTA with both filter tables staged, when that keeps as many CTAs per
      // SM as 32 features without the w' table (which then comes from global memory)
      const MsgSmem l16 = msg_smem_layout<T>(d.N, IB, CB, true, 16);
      auto per_sm = [](int bytes) { return (228 * 1024) / (bytes + 1024); };
      if (l16.total_bytes <= 220 * 1024 && per_sm(l16.total_bytes) >= per_sm(lay.total_bytes)) {
        stage_w1 = true;
        L = 16;
        lay = l16;
      }
    }
    if (lay.total_bytes > 220 * 1024) {
      L = 16;
      lay = msg_smem_layout<T>(d.N, IB, CB, stage_w1, L);
    }
    if (lay.total_bytes > 220 * 1024) return cudaErrorInvalidConfiguration;
    smem = std::max(smem, lay.total_bytes);
    ent[ne++] = Ent{{m[k].b.Z, m[k].b.z0, m[k].b.ew, m[k].b.geo, m[k].params + h.off.layer[l].Y, h.d_pair_of, d.N,
                     d.n_up, d.M, d.C, d.D, h.edges.n_all, h.edges.n_ee, z_const && !h.el_init ? 1 : 0, stage_w1 ? 1 : 0,
                     out_of(m[k])},
                    d.Bc, d.D / L, L, lay.total_bytes, 0};
  }
  if (ne == 0) return cudaSuccess;
  auto kern = messages_kernel_group<T, TO, IB, CB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  // One launch per occupancy class: molecules whose CTAs fit the same number per SM share a
  // launch (the launch's shared memory is its largest entry's, which sets everyone's occupancy).
  for (int i = 0; i < ne; ++i) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ent[i].occ, kern, 32 * kMsgWarps, ent[i].smem);
    if (e != cudaSuccess) return e;
  }
  bool done[kMaxGroup] = {};
  for (int i = 0; i < ne; ++i) {
    if (done[i]) continue;
    Grp<messages_kernel_args<T, TO>> g{};
    int sm = 0;
    for (int j = i; j < ne; ++j)
      if (!done[j] && ent[j].occ == ent[i].occ) {
        g.add(ent[j].a, ent[j].bx, ent[j].ny, ent[j].L);
        sm = std::max(sm, ent[j].smem);
        done[j] = true;
      }
    e = check_group(g);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)g.blocks(), 32 * kMsgWarps, sm, s>>>(g);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
}  // namespace

template <class T>
cudaError_t launch_messages_group(const MolFwd<T>* m, int n, int l, bool z_const, cudaStream_t s) {
  if (n > kMaxGroup) return cudaErrorInvalidValue;
  if (n == 0) return cudaSuccess;
  // receivers per warp task (the register tile IB x CB): the handle's tuned value, else the default
  if constexpr (sizeof(T) == 4) {
    const bool ib4 = m[0].h->msg_ib == 4;
    if (m[0].b.msg_bf)
      return ib4 ? launch_messages_group_t<T, __nv_bfloat16, 4>(m, n, l, z_const, true, s)
                 : launch_messages_group_t<T, __nv_bfloat16, 8>(m, n, l, z_const, true, s);
    return ib4 ? launch_messages_group_t<T, T, 4>(m, n, l, z_const, false, s)
               : launch_messages_group_t<T, T, 8>(m, n, l, z_const, false, s);
  }
  return launch_messages_group_t<T, T, msg_ib<T>()>(m, n, l, z_const, false, s);
}

template <class T>
cudaError_t launch_update_group(const MolFwd<T>* m, int n, bool from_spin, cudaStream_t s) {
  if (n > kMaxGroup) return cudaErrorInvalidValue;
  Grp<update_kernel_args<T>> g{};
  for (int k = 0; k < n; ++k) {
    const FwdDims& d = m[k].d;
    if (d.Bc <= 0) continue;
    g.add({m[k].b.Z, m[k].b.F, m[k].b.F, m[k].params + std::max<int64_t>(m[k].h->off.E_spin, 0), d.Bc, d.N, d.n_up, d.C, d.D,
           from_spin && !m[k].h->el_init ? 1 : 0, static_cast<__nv_bfloat16*>(m[k].b.F_bf)},
          blocks(d.Bc * d.N * d.D, 256));
  }
  if (g.n == 0) return cudaSuccess;
  cudaError_t e = check_group(g);
  if (e != cudaSuccess) return e;
  update_kernel_group<T><<<(unsigned)g.blocks(), 256, 0, s>>>(g);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_orbital_det_group(const MolFwd<T>* m, int n, cudaStream_t s) {
  if (n > kMaxGroup) return cudaErrorInvalidValue;
  struct Ent {
    orbital_det_kernel_args<T> a;
    int64_t bx;
    int tag, occ;
    size_t smem;
  };
  Ent ent[kMaxGroup];
  int ne = 0;
  size_t smem = 0;
  // warps (one matrix each) per CTA, one choice for the launch: the first handle's
  const int W = (n > 0 && m[0].h->det_warps == 2) ? 2 : 4;
  for (int k = 0; k < n; ++k) {
    const dq_handle_s& h = *m[k].h;
    const FwdDims& d = m[k].d;
    if (d.Bc <= 0) continue;
    const int nmax = h.det_n();
    const int64_t nmat = d.Bc * 2 * d.K;
    size_t sm4 = 0;
    const int tag = det_body_tag<T>(nmax, d.N, d.C, &sm4);
    if (tag == 0 && sm4 > 200 * 1024) return cudaErrorInvalidConfiguration;  // grouped form: four warps per CTA
    const size_t sm = sm4 / 4 * W;
    smem = std::max(smem, sm);
    ent[ne++] = Ent{{m[k].b.phi, m[k].b.geo, m[k].params, d.Bc, d.N, d.n_up, d.M, d.K, d.C, d.K * nmax,
                     h.edges.n_all, h.edges.n_ee, h.off.omega[0], h.off.omega[1], h.off.zeta[0], h.off.zeta[1],
                     m[k].b.det, h.d_fp64_count, h.full_det},
                    blocks(nmat, W), tag, 0, sm};
  }
  if (ne == 0) return cudaSuccess;
  // kernel of each body: 0 the mixed / general group kernel, 1 and 2 the large-block ones
  auto kind = [](int tag) { return tag == 2 ? 1 : tag == 3 ? 2 : 0; };
  const void* kerns[3] = {nullptr, nullptr, nullptr};
  if constexpr (sizeof(T) == 4) {
    kerns[0] = (const void*)orbital_det_mixed_group;
    kerns[1] = (const void*)orbital_det_large_group<16>;
    kerns[2] = (const void*)orbital_det_large_group<kDetNRL>;
  } else {
    kerns[0] = (const void*)orbital_det_kernel_group<T>;
  }
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < ne; ++i) {
    e = cudaFuncSetAttribute(kerns[kind(ent[i].tag)], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // one launch per kernel and occupancy class (see launch_messages_group)
  for (int i = 0; i < ne; ++i) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ent[i].occ, kerns[kind(ent[i].tag)], 32 * W, ent[i].smem);
    if (e != cudaSuccess) return e;
  }
  bool done[kMaxGroup] = {};
  for (int i = 0; i < ne; ++i) {
    if (done[i]) continue;
    Grp<orbital_det_kernel_args<T>> g{};
    size_t sm = 0;
    const int k = kind(ent[i].tag);
    for (int j = i; j < ne; ++j)
      if (!done[j] && ent[j].occ == ent[i].occ && kind(ent[j].tag) == k) {
        g.add(ent[j].a, ent[j].bx, 1, ent[j].tag);
        sm = std::max(sm, ent[j].smem);
        done[j] = true;
      }
    e = check_group(g);
    if (e != cudaSuccess) return e;
    if constexpr (sizeof(T) == 4) {
      if (k == 1) orbital_det_large_group<16><<<(unsigned)g.blocks(), 32 * W, sm, s>>>(g);
      else if (k == 2) orbital_det_large_group<kDetNRL><<<(unsigned)g.blocks(), 32 * W, sm, s>>>(g);
      else orbital_det_mixed_group<<<(unsigned)g.blocks(), 32 * W, sm, s>>>(g);
    } else {
      orbital_det_kernel_group<T><<<(unsigned)g.blocks(), 32 * W, sm, s>>>(g);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class T>
cudaError_t launch_jastrow_sum_group(const MolFwd<T>* m, int n, cudaStream_t s) {
  if (n > kMaxGroup) return cudaErrorInvalidValue;
  Grp<jastrow_sum_kernel_args<T>> g{};
  for (int k = 0; k < n; ++k) {
    const FwdDims& d = m[k].d;
    if (d.Bc <= 0 || !m[k].h->use_jastrow) continue;
    g.add({m[k].b.F, d.Bc, d.N, d.C, d.D, m[k].b.js}, blocks(d.Bc * d.C * d.D, 256));
  }
  if (g.n == 0) return cudaSuccess;
  cudaError_t e = check_group(g);
  if (e != cudaSuccess) return e;
  jastrow_sum_kernel_group<T><<<(unsigned)g.blocks(), 256, 0, s>>>(g);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_combine_group(const MolFwd<T>* m, int n, T* const* logabs, int8_t* const* sign, T* const* e_loc,
                                 T* const* grad, cudaStream_t s) {
  if (n > kMaxGroup) return cudaErrorInvalidValue;
  Grp<combine_kernel_args<T>> g{};
  size_t smem = 0;
  for (int k = 0; k < n; ++k) {
    const dq_handle_s& h = *m[k].h;
    const FwdDims& d = m[k].d;
    if (d.Bc <= 0) continue;
    smem = std::max(smem, (2 * (size_t)d.K + 3 * (size_t)d.D + 32 + 3 * (size_t)d.N) * sizeof(double));
    g.add({m[k].b.det, m[k].b.jh, m[k].b.geo, m[k].params, h.d_Z, h.d_pair_ij, h.d_pair_of, d.Bc, d.N, d.n_up, d.M,
           d.K, d.C, d.D, h.edges.n_all, h.edges.n_ee, h.off.c, h.off.w_J2, h.use_jastrow, h.use_cusp, h.alpha, h.Vnn,
           logabs[k], sign[k], e_loc ? e_loc[k] : nullptr, grad ? grad[k] : nullptr, h.d_status},
          d.Bc);
  }
  if (g.n == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(combine_kernel_group<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  combine_kernel_group<T><<<(unsigned)g.blocks(), kCombineThreads, smem, s>>>(g);
  return cudaGetLastError();
}

#define DQ_INSTANTIATE_GROUP(T)                                                                                    \
  template cudaError_t launch_geometry_group<T>(const MolFwd<T>*, int, const T* const*, cudaStream_t);            \
  template cudaError_t launch_edge_hidden_group<T>(const MolFwd<T>*, int, int, cudaStream_t);                     \
  template cudaError_t launch_edge_update_group<T>(const MolFwd<T>*, int, int, const T* const*, T* const*,         \
                                                   cudaStream_t);                                                 \
  template cudaError_t launch_edge_update<T>(const dq_handle_s&, const FwdDims&, const T*, int, const T*, T*,      \
                                             cudaStream_t);                                                       \
  template cudaError_t launch_el_init<T>(const dq_handle_s&, const FwdDims&, const T*, const T*, T*, void*, T*, T*, \
                                         cudaStream_t);                                                           \
  template cudaError_t launch_layer0_node_group<T>(const MolFwd<T>*, int, cudaStream_t);                          \
  template cudaError_t launch_messages_group<T>(const MolFwd<T>*, int, int, bool, cudaStream_t);                  \
  template cudaError_t launch_update_group<T>(const MolFwd<T>*, int, bool, cudaStream_t);                         \
  template cudaError_t launch_orbital_det_group<T>(const MolFwd<T>*, int, cudaStream_t);                          \
  template cudaError_t launch_jastrow_sum_group<T>(const MolFwd<T>*, int, cudaStream_t);                          \
  template cudaError_t launch_combine_group<T>(const MolFwd<T>*, int, T* const*, int8_t* const*, T* const*,      \
                                               T* const*, cudaStream_t);
DQ_INSTANTIATE_GROUP(float)
DQ_INSTANTIATE_GROUP(double)

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
  template cudaError_t launch_update_io<T>(const dq_handle_s&, const FwdDims&, const T*, bool, const T*, const T*, \
                                           T*, cudaStream_t, void*);                                              \
  template cudaError_t launch_orbital_det<T>(const dq_handle_s&, const FwdDims&, const T*, FwdBuffers<T>,         \
                                             cudaStream_t);                                                       \
  template cudaError_t launch_jastrow_sum<T>(const dq_handle_s&, const FwdDims&, FwdBuffers<T>, cudaStream_t);    \
  template cudaError_t launch_combine<T>(const dq_handle_s&, const FwdDims&, const T*, FwdBuffers<T>, T*,         \
                                         int8_t*, T*, cudaStream_t, T*);

DQ_INSTANTIATE(float)
DQ_INSTANTIATE(double)

}  // namespace dq
