// Natural-gradient direction of the optimiser (Sec. 4, "Optimizer"): the loss
// gradient g = G^T w of Eq. (30) preconditioned by the damped Fisher information
// of |psi|^2 estimated from the walkers,
//   delta = (Gc^T Gc / B + lambda I)^-1 g = Gc^T (Gc Gc^T / B + lambda I)^-1 w,
// Gc = G - mean over walkers.  The second (sample-space) form needs a B x B
// system only: the Gram matrix Gc Gc^T comes from the 3 x TF32 tensor-core GEMM
// (gemm_tc.cu), the system is solved by conjugate gradients preconditioned with
// its diagonal (walkers' gradient norms span orders of magnitude near the
// nodes), in FP64 with fixed-order reductions (deterministic), and delta =
// Gc^T x is a weighted column sum.  The conjugate-gradient loop runs as a fixed sequence of launches
// that stop working once a flag in device memory says the residual is small
// enough, so the whole call can be captured in a CUDA graph.
#include <math.h>

#include "common.cuh"

namespace dq {
namespace {

constexpr int kNgThreads = 256;
constexpr int64_t kNgChunk = 8192;  // K extent of one Gram chunk (FP32 accumulation length)
constexpr int kNgJobs = 16;         // chunks per GEMM launch
constexpr int kNgRowWarps = 8;  // matvec: one warp per row of the Gram matrix

// mean[p] = (1 / B) sum_b G[b][p], in FP64, one thread per column (fixed order over b)
__global__ void ng_colmean_kernel(const float* __restrict__ G, int64_t B, int64_t P, double* __restrict__ mean) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double s = 0;
  for (int64_t b = 0; b < B; ++b) s += (double)G[b * P + p];
  mean[p] = s / (double)B;
}

// Gc[b][p] = G[b][p] - mean[p] with row pitch Pp (zeros in the padding)
__global__ void ng_center_kernel(const float* __restrict__ G, const double* __restrict__ mean, int64_t B, int64_t P,
                                 int64_t Pp, float* __restrict__ Gc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * Pp) return;
  const int64_t b = e / Pp, p = e - (e / Pp) * Pp;
  Gc[e] = p < P ? (float)((double)G[b * P + p] - mean[p]) : 0.f;
}

struct CgScalars {
  double rr, rr0, rz, pAp, beta, lam;
  double tol2;  // (tol ||w||)^2
  int iter, max_iter, done, pad;
  unsigned int counter;  // arrivals of the CTAs of the current reduction
};

// Block sum in FP64, fixed order (tree over the block's threads).
__device__ double ng_block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Last-arriving CTA adds the per-CTA partials in index order; returns true in that CTA
// (the sum is then in *out).
__device__ bool ng_finish(double part, double* partials, unsigned int* counter, double* out) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = part;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __shared__ double sh[kNgThreads];
  double s = 0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += ((volatile double*)partials)[i];
  // fixed order: strided per thread, then the block tree
  s = ng_block_sum(s, sh);
  if (threadIdx.x == 0) {
    *out = s;
    *counter = 0;
  }
  return true;
}

// x = 0, r = w, p = z = r / diag(A), rr = rr0 = r.r, rz = r.z (one CTA)
__global__ void ng_cg_init_kernel(const float* __restrict__ w, int64_t B, const double* __restrict__ T, double* x,
                                  double* r, double* p, double* dinv, CgScalars* sc, double lam, double tol,
                                  int max_iter) {
  __shared__ double sh[kNgThreads];
  if (lam < 0) {  // relative damping: |lam| x the mean eigenvalue tr(T) / B^2 of T / B
    double tr = 0;
    for (int64_t i = threadIdx.x; i < B; i += blockDim.x) tr += T[i * B + i];
    tr = ng_block_sum(tr, sh);
    lam = -lam * tr / ((double)B * (double)B);
    if (!(lam > 0)) lam = 1.0;  // all-zero gradients: any positive damping gives delta = 0
  }
  double s = 0, sz = 0;
  for (int64_t i = threadIdx.x; i < B; i += blockDim.x) {
    const double v = (double)w[i];
    const double di = 1.0 / (T[i * B + i] / (double)B + lam);
    dinv[i] = di;
    x[i] = 0;
    r[i] = v;
    p[i] = v * di;
    s += v * v;
    sz += v * v * di;
  }
  s = ng_block_sum(s, sh);
  sz = ng_block_sum(sz, sh);
  if (threadIdx.x == 0) {
    sc->rr = s;
    sc->rr0 = s;
    sc->rz = sz;
    sc->pAp = 0;
    sc->beta = 0;
    sc->lam = lam;
    sc->tol2 = tol * tol * s;
    sc->iter = 0;
    sc->max_iter = max_iter;
    sc->done = s == 0.0 || max_iter <= 0;
    sc->counter = 0;
  }
}

// T (+)= sum of the chunks' Gram matrices, in FP64 and chunk order
__global__ void ng_gram_add_kernel(const float* __restrict__ Tc, int n_chunks, int64_t BB, int first,
                                   double* __restrict__ T) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= BB) return;
  double s = first ? 0.0 : T[e];
  for (int c = 0; c < n_chunks; ++c) s += (double)Tc[(int64_t)c * BB + e];
  T[e] = s;
}

// T = (T + T^T) / 2: the 3 x TF32 products of T_ij and T_ji drop different low-order
// terms, and conjugate gradients need an exactly symmetric matrix
__global__ void ng_symmetrize_kernel(double* T, int64_t B) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * B) return;
  const int64_t i = e / B, j = e - (e / B) * B;
  if (j <= i) return;
  const double a = 0.5 * (T[i * B + j] + T[j * B + i]);
  T[i * B + j] = a;
  T[j * B + i] = a;
}

// Ap = T p / B + lam p and pAp = p . Ap; one warp per row of T (B x B, FP64)
__global__ void __launch_bounds__(32 * kNgRowWarps)
    ng_cg_matvec_kernel(const double* __restrict__ T, int64_t B, const double* __restrict__ p, double* __restrict__ Ap,
                        CgScalars* sc, double* partials) {
  if (((volatile CgScalars*)sc)->done) return;
  const int lane = threadIdx.x % 32, wq = threadIdx.x / 32;
  const int64_t i = (int64_t)blockIdx.x * kNgRowWarps + wq;
  double part = 0;
  if (i < B) {
    const double* Ti = T + i * B;
    double s = 0;
    for (int64_t j = lane; j < B; j += 32) s += Ti[j] * p[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double a = s / (double)B + sc->lam * p[i];
    if (lane == 0) Ap[i] = a;
    part = lane == 0 ? a * p[i] : 0.0;
  }
  __shared__ double sh[32 * kNgRowWarps];
  const double cta = ng_block_sum(part, sh);
  ng_finish(cta, partials, &sc->counter, &sc->pAp);
}

// alpha = rz / pAp; x += alpha p; r -= alpha Ap; z = r / diag(A); rr' = r.r, rz' = r.z;
// beta = rz' / rz; convergence flag (on ||r|| / ||w||)
__global__ void ng_cg_update_kernel(int64_t B, double* x, double* r, double* z, const double* __restrict__ dinv,
                                    const double* __restrict__ p, const double* __restrict__ Ap, CgScalars* sc,
                                    double* partials, double* partials2) {
  volatile CgScalars* vs = sc;
  if (vs->done) return;
  const double alpha = vs->pAp > 0 ? vs->rz / vs->pAp : 0.0;
  double part = 0, partz = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * Ap[i];
    const double zi = ri * dinv[i];
    r[i] = ri;
    z[i] = zi;
    part += ri * ri;
    partz += ri * zi;
  }
  __shared__ double sh[kNgThreads];
  const double cta = ng_block_sum(part, sh);
  const double ctaz = ng_block_sum(partz, sh);
  if (threadIdx.x == 0) partials2[blockIdx.x] = ctaz;  // published before this CTA's arrival in ng_finish
  double rr_new = 0;
  if (ng_finish(cta, partials, &sc->counter, &rr_new)) {
    __shared__ double shz[kNgThreads];
    double s = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += ((volatile double*)partials2)[i];
    const double rz_new = ng_block_sum(s, shz);
    if (threadIdx.x == 0) {
      const int it = vs->iter;
      sc->beta = vs->rz > 0 ? rz_new / vs->rz : 0.0;
      sc->rz = rz_new;
      sc->rr = rr_new;
      sc->iter = it + 1;
      sc->done = (rr_new <= vs->tol2 || it + 1 >= vs->max_iter || !(vs->pAp > 0)) ? 1 : 0;
    }
  }
}

// p = z + beta p
__global__ void ng_cg_direction_kernel(int64_t B, const double* __restrict__ z, double* p, const CgScalars* sc) {
  const volatile CgScalars* vs = sc;
  if (vs->done) return;
  const double beta = vs->beta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// delta[p] = sum_b x_b Gc[b][p] (fixed order over b); stats
__global__ void ng_apply_kernel(const float* __restrict__ Gc, int64_t B, int64_t P, int64_t Pp,
                                const double* __restrict__ x, float* __restrict__ delta) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P) return;
  double s = 0;
  for (int64_t b = 0; b < B; ++b) s += x[b] * (double)Gc[b * Pp + q];
  delta[q] = (float)s;
}

__global__ void ng_stats_kernel(const CgScalars* sc, double* stats) {
  stats[0] = (double)sc->iter;
  stats[1] = sc->rr0 > 0 ? sqrt(sc->rr / sc->rr0) : 0.0;
  stats[2] = sqrt(sc->rr0);
  stats[3] = sc->lam;
}

inline unsigned ng_blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
inline size_t ng_align(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

// Workspace layout of natgrad_run (bytes), for B walkers and P parameters.
size_t natgrad_workspace(int64_t B, int64_t P) {
  const int64_t Pp = (P + 3) / 4 * 4;
  const int64_t mv_ctas = (B + kNgRowWarps - 1) / kNgRowWarps;
  size_t o = 0;
  o += ng_align((size_t)P * 8);                 // mean
  o += 3 * ng_align((size_t)B * Pp * 4);        // Gc, TF32 high, TF32 low
  o += ng_align((size_t)kNgJobs * B * B * 4);  // Gram matrices of the chunks of one launch
  o += ng_align((size_t)B * B * 8);             // Gram matrix (FP64)
  o += 6 * ng_align((size_t)B * 8);             // x, r, p, Ap, z, 1 / diag
  o += 2 * ng_align((size_t)(mv_ctas + 1024) * 8);  // partials
  o += ng_align(sizeof(CgScalars));
  return o;
}

cudaError_t natgrad_run(const float* G, const float* w, int64_t B, int64_t P, double lam, int max_iter, double tol,
                        float* delta, double* stats, unsigned char* ws, unsigned int* status, cudaStream_t s) {
  const int64_t Pp = (P + 3) / 4 * 4;
  const int64_t mv_ctas = (B + kNgRowWarps - 1) / kNgRowWarps;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    unsigned char* q = ws + o;
    o += ng_align(bytes);
    return q;
  };
  double* mean = reinterpret_cast<double*>(take((size_t)P * 8));
  float* Gc = reinterpret_cast<float*>(take((size_t)B * Pp * 4));
  float* Wb = reinterpret_cast<float*>(take((size_t)B * Pp * 4));
  float* Wsm = reinterpret_cast<float*>(take((size_t)B * Pp * 4));
  float* Tc = reinterpret_cast<float*>(take((size_t)kNgJobs * B * B * 4));
  double* T = reinterpret_cast<double*>(take((size_t)B * B * 8));
  double* x = reinterpret_cast<double*>(take((size_t)B * 8));
  double* r = reinterpret_cast<double*>(take((size_t)B * 8));
  double* p = reinterpret_cast<double*>(take((size_t)B * 8));
  double* Ap = reinterpret_cast<double*>(take((size_t)B * 8));
  double* z = reinterpret_cast<double*>(take((size_t)B * 8));
  double* dinv = reinterpret_cast<double*>(take((size_t)B * 8));
  double* partials = reinterpret_cast<double*>(take((size_t)(mv_ctas + 1024) * 8));
  double* partials2 = reinterpret_cast<double*>(take((size_t)(mv_ctas + 1024) * 8));
  CgScalars* sc = reinterpret_cast<CgScalars*>(take(sizeof(CgScalars)));

  ng_colmean_kernel<<<ng_blocks(P, kNgThreads), kNgThreads, 0, s>>>(G, B, P, mean);
  ng_center_kernel<<<ng_blocks(B * Pp, kNgThreads), kNgThreads, 0, s>>>(G, mean, B, P, Pp, Gc);
  cudaError_t e = split_tf32(Gc, Wb, Wsm, B * Pp, s);
  if (e != cudaSuccess) return e;
  // T = Gc Gc^T (B x B): rows of Gc against the TF32 parts of Gc, in chunks of kNgChunk
  // columns (each accumulated in FP32 on the tensor cores), the chunks added in FP64
  const int64_t n_chunks = (Pp + kNgChunk - 1) / kNgChunk;
  for (int64_t c0 = 0; c0 < n_chunks; c0 += kNgJobs) {
    T3JobDesc jd[kNgJobs];
    int nj = 0;
    for (int64_t c = c0; c < n_chunks && nj < kNgJobs; ++c, ++nj) {
      const int64_t k0 = c * kNgChunk, kc = Pp - k0 < kNgChunk ? Pp - k0 : kNgChunk;
      jd[nj] = T3JobDesc{Gc + k0, B, 1, 0, (int)kc, Pp, Wb + k0, Wsm + k0, (int)B, nullptr, 1,
                         Tc + (int64_t)nj * B * B, B, 0, false, Pp};
    }
    e = gemm_tf32x3_tc_jobs(jd, nj, status, s);
    if (e != cudaSuccess) return e;
    ng_gram_add_kernel<<<ng_blocks(B * B, kNgThreads), kNgThreads, 0, s>>>(Tc, nj, B * B, c0 == 0 ? 1 : 0, T);
  }
  ng_symmetrize_kernel<<<ng_blocks(B * B, kNgThreads), kNgThreads, 0, s>>>(T, B);
  ng_cg_init_kernel<<<1, kNgThreads, 0, s>>>(w, B, T, x, r, p, dinv, sc, lam, tol, max_iter);
  const unsigned up_ctas = ng_blocks(B, kNgThreads) < 1024 ? ng_blocks(B, kNgThreads) : 1024;
  for (int it = 0; it < max_iter; ++it) {
    ng_cg_matvec_kernel<<<(unsigned)mv_ctas, 32 * kNgRowWarps, 0, s>>>(T, B, p, Ap, sc, partials);
    ng_cg_update_kernel<<<up_ctas, kNgThreads, 0, s>>>(B, x, r, z, dinv, p, Ap, sc, partials, partials2);
    ng_cg_direction_kernel<<<up_ctas, kNgThreads, 0, s>>>(B, z, p, sc);
  }
  ng_apply_kernel<<<ng_blocks(P, kNgThreads), kNgThreads, 0, s>>>(Gc, B, P, Pp, x, delta);
  if (stats) ng_stats_kernel<<<1, 1, 0, s>>>(sc, stats);
  return cudaGetLastError();
}

}  // namespace dq

namespace dq {
namespace {
// ||delta||^2 in FP64: per-CTA partials, the last CTA adds them in index order and
// sets the step scale s = min(1, max_norm / (lr ||delta||)) (no limit when max_norm <= 0)
__global__ void ng_norm_kernel(const float* __restrict__ d, int64_t P, double lr, double max_norm,
                               double* partials, unsigned int* counter, double* out) {
  double part = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)d[i];
    part += v * v;
  }
  __shared__ double sh[kNgThreads];
  const double cta = ng_block_sum(part, sh);
  double ss = 0;
  if (ng_finish(cta, partials, counter, &ss) && threadIdx.x == 0) {
    const double nrm = sqrt(ss);
    out[0] = nrm;
    out[1] = (max_norm > 0 && lr * nrm > max_norm) ? max_norm / (lr * nrm) : 1.0;
  }
}

// theta -= lr * s * delta
template <class T>
__global__ void ng_update_kernel(T* __restrict__ theta, const T* __restrict__ d, int64_t P, double lr,
                                 const double* __restrict__ nrm) {
  const double step = lr * nrm[1];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
    theta[i] = (T)((double)theta[i] - step * (double)d[i]);
}
}  // namespace

size_t param_update_workspace() { return 1024 * 8 + 256; }

template <class T>
cudaError_t param_update_run(T* theta, const T* delta, int64_t P, double lr, double max_norm, double* stats,
                             unsigned char* ws, cudaStream_t s) {
  double* partials = reinterpret_cast<double*>(ws);
  unsigned int* counter = reinterpret_cast<unsigned int*>(ws + 1024 * 8);
  const unsigned ctas = ng_blocks(P, kNgThreads) < 1024 ? ng_blocks(P, kNgThreads) : 1024;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  if constexpr (sizeof(T) == 4) {
    ng_norm_kernel<<<ctas, kNgThreads, 0, s>>>(delta, P, lr, max_norm, partials, counter, stats);
  } else {
    return cudaErrorInvalidValue;  // FP32 modes only
  }
  ng_update_kernel<T><<<ctas, kNgThreads, 0, s>>>(theta, delta, P, lr, stats);
  return cudaGetLastError();
}
template cudaError_t param_update_run<float>(float*, const float*, int64_t, double, double, double*, unsigned char*,
                                             cudaStream_t);

}  // namespace dq
