// Local and non-local pseudopotential energies (Eqs. 11 and 12).
// For walker b, electron i and a nucleus I that carries a
// pseudopotential, the non-local term is
//   sum_l W_l(r_iI) (2l + 1) / 12 sum_k P_l(cos th_k) psi(r_i -> R_I + r_iI R_b u_k) / psi(r),
// the addition theorem turning the sum over m of Y_lm(Omega) Y_lm^*(Omega')
// into (2l + 1) / (4 pi) P_l(cos), and the 12-point icosahedral rule (vertices
// u_k rotated by the walker's rotation R_b) replacing int dOmega' by
// (4 pi / 12) sum_k; cos th_k = (R_b u_k) . (r_i - R_I) / r_iI.  Radial
// functions f(r) = sum_t beta_t r^(n_t - 2) exp(-alpha_t r^2); the local part is
// sum_{i,I} V_I(r_iI).  The psi ratios come from the value-only forward pass on
// all displaced configurations (one batch), combined in FP64.
#include <math.h>

#include "common.cuh"

namespace dq {
namespace {

__device__ __forceinline__ void pp_vertex(int k, double R9[9], double out[3]) {
  // vertices in the order (0, a, b), (a, b, 0), (b, 0, a) for a = -1, 1 and b = -g, g
  const double g = 0.5 * (1.0 + sqrt(5.0));
  const int ia = k / 6, ib = (k / 3) % 2, c = k % 3;
  const double a = ia ? 1.0 : -1.0, bb = ib ? g : -g;
  double v[3];
  if (c == 0) { v[0] = 0; v[1] = a; v[2] = bb; }
  else if (c == 1) { v[0] = a; v[1] = bb; v[2] = 0; }
  else { v[0] = bb; v[1] = 0; v[2] = a; }
  const double nrm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int x = 0; x < 3; ++x) out[x] = (R9[3 * x] * v[0] + R9[3 * x + 1] * v[1] + R9[3 * x + 2] * v[2]) / nrm;
}

__device__ __forceinline__ double pp_radial_d(const PPSet& pp, int q, int chan, double r) {
  double s = 0;
  const int base = (q * (kMaxPPChan) + chan) * kMaxPPTerms;
  for (int t = 0; t < pp.n_terms[q]; ++t) {
    const double be = pp.c[base + t][0], n = pp.c[base + t][1], al = pp.c[base + t][2];
    s += be * pow(r, n - 2.0) * exp(-al * r * r);
  }
  return s;
}

__device__ __forceinline__ double pp_legendre(int l, double x) {
  return l == 0 ? 1.0 : l == 1 ? x : l == 2 ? 0.5 * (3 * x * x - 1) : 0.5 * (5 * x * x * x - 3 * x);
}

// configs[b][pair][k][j][x], pair = i * n_pp + q: walker b with electron i moved to
// R_I + r_iI R_b u_k (I = nucleus of pseudopotential q)
template <class T>
__global__ void pp_displace_kernel(const T* __restrict__ r, const double* __restrict__ Rn, const T* __restrict__ rot,
                                   int64_t B, int N, const __grid_constant__ PPSet pp, T* __restrict__ configs) {
  const int npairs = N * pp.n;
  const int64_t per = (int64_t)npairs * 12 * N * 3;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * per) return;
  const int64_t b = e / per;
  int64_t rem = e - b * per;
  const int pair = (int)(rem / (12 * N * 3));
  rem -= (int64_t)pair * 12 * N * 3;
  const int k = (int)(rem / (N * 3));
  rem -= (int64_t)k * N * 3;
  const int j = (int)(rem / 3), x = (int)(rem % 3);
  const int i = pair / pp.n, q = pair % pp.n, I = pp.nucleus[q];
  const T* rb = r + b * N * 3;
  if (j != i) {
    configs[e] = rb[j * 3 + x];
    return;
  }
  double d[3];
  for (int y = 0; y < 3; ++y) d[y] = (double)rb[i * 3 + y] - Rn[I * 3 + y];
  const double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double R9[9], u[3];
  for (int y = 0; y < 9; ++y) R9[y] = (double)rot[b * 9 + y];
  pp_vertex(k, R9, u);
  configs[e] = (T)(Rn[I * 3 + x] + rr * u[x]);
}

// one warp per walker: v_loc = sum_{i,q} V_q(r_iI), v_nl = sum_{i,q,k} w_iqk psi'/psi
template <class T>
__global__ void pp_combine_kernel(const T* __restrict__ r, const double* __restrict__ Rn, const T* __restrict__ rot,
                                  const T* __restrict__ logabs, const int8_t* __restrict__ sign,
                                  const T* __restrict__ la_c, const int8_t* __restrict__ sg_c, int64_t B, int N,
                                  const __grid_constant__ PPSet pp, T* __restrict__ v_loc, T* __restrict__ v_nl) {
  const int lane = threadIdx.x % 32;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (b >= B) return;
  const int npairs = N * pp.n, items = npairs * 12;
  const T* rb = r + b * N * 3;
  double R9[9];
  for (int y = 0; y < 9; ++y) R9[y] = (double)rot[b * 9 + y];
  const double la0 = (double)logabs[b];
  const int s0 = sign[b];
  double snl = 0, sloc = 0;
  for (int it = lane; it < items; it += 32) {
    const int pair = it / 12, k = it % 12;
    const int i = pair / pp.n, q = pair % pp.n, I = pp.nucleus[q];
    double d[3];
    for (int y = 0; y < 3; ++y) d[y] = (double)rb[i * 3 + y] - Rn[I * 3 + y];
    const double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double u[3];
    pp_vertex(k, R9, u);
    const double cs = (u[0] * d[0] + u[1] * d[1] + u[2] * d[2]) / rr;
    double w = 0;
    for (int l = 0; l <= pp.lmax[q]; ++l) w += pp_radial_d(pp, q, 1 + l, rr) * (2 * l + 1) / 12.0 * pp_legendre(l, cs);
    const int64_t c = b * items + it;
    const double ratio = (double)(sg_c[c] * s0) * exp((double)la_c[c] - la0);
    snl += w * ratio;
    if (k == 0) sloc += pp_radial_d(pp, q, 0, rr);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    snl += __shfl_xor_sync(0xffffffffu, snl, o);
    sloc += __shfl_xor_sync(0xffffffffu, sloc, o);
  }
  if (lane == 0) {
    v_nl[b] = (T)snl;
    v_loc[b] = (T)sloc;
  }
}

inline unsigned pp_blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

template <class T>
cudaError_t pp_displace(const T* r, const double* Rn, const T* rot, int64_t B, int N, const PPSet& pp, T* configs,
                        cudaStream_t s) {
  const int64_t n = B * (int64_t)N * pp.n * 12 * N * 3;
  pp_displace_kernel<T><<<pp_blocks(n, 256), 256, 0, s>>>(r, Rn, rot, B, N, pp, configs);
  return cudaGetLastError();
}

template <class T>
cudaError_t pp_combine(const T* r, const double* Rn, const T* rot, const T* logabs, const int8_t* sign, const T* la_c,
                       const int8_t* sg_c, int64_t B, int N, const PPSet& pp, T* v_loc, T* v_nl, cudaStream_t s) {
  pp_combine_kernel<T><<<pp_blocks(B, 8), 256, 0, s>>>(r, Rn, rot, logabs, sign, la_c, sg_c, B, N, pp, v_loc, v_nl);
  return cudaGetLastError();
}

#define DQ_PP_INST(T)                                                                                              \
  template cudaError_t pp_displace<T>(const T*, const double*, const T*, int64_t, int, const PPSet&, T*,            \
                                      cudaStream_t);                                                              \
  template cudaError_t pp_combine<T>(const T*, const double*, const T*, const T*, const int8_t*, const T*,         \
                                     const int8_t*, int64_t, int, const PPSet&, T*, T*, cudaStream_t);
DQ_PP_INST(float)
DQ_PP_INST(double)

}  // namespace dq
