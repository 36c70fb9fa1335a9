// Random-walk Metropolis sampler (Sec. 5), FP64 walker-sum of local energies
// and the clipped-energy weights of the gradient estimator (Sec. 4.4, Eq. 30).
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written
// from its published definition: ten rounds of two 32x32->64-bit products with
// multipliers 0xD2511F53 and 0xCD9E8D57, key schedule bumped by the Weyl
// constants 0x9E3779B9 and 0xBB67AE85.  Counter [walker, t_lo, (tag << 24) |
// block, t_hi], key [seed_lo, seed_hi]; uniforms (x + 0.5) 2^-32; normals by
// Box-Muller in FP64 from the word pairs (x0, x1) and (x2, x3).
#include <math.h>

#include "common.cuh"

namespace dq {
namespace {

constexpr uint32_t kTagPropose = 1, kTagAccept = 2;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ double unit_uniform(uint32_t x) { return ((double)x + 0.5) * 2.3283064365386963e-10; }

template <class T>
struct propose_kernel_args {
  const T* r;
  T* r_prop;
  int64_t B;
  int N3;
  double step;
  uint64_t seed;
  uint64_t t;
  const uint64_t* t_base;
};

template <class T>
__device__ __forceinline__ void propose_kernel_body(const int64_t bx_, const int by_, const int64_t nbx_, const T* __restrict__ r, T* __restrict__ r_prop, int64_t B, int N3, double step,
                               uint64_t seed, uint64_t t, const uint64_t* __restrict__ t_base) {
  if (t_base) t += *t_base;  // step counter kept in device memory
  const int nblk = (N3 + 3) / 4;
  const int64_t gid = (int64_t)bx_ * blockDim.x + threadIdx.x;
  if (gid >= B * nblk) return;
  const int64_t b = gid / nblk;
  const int blk = (int)(gid % nblk);
  const uint4 ctr = make_uint4((uint32_t)b, (uint32_t)t, (kTagPropose << 24) | (uint32_t)blk, (uint32_t)(t >> 32));
  const uint4 x = philox4x32_10(ctr, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const double ra = sqrt(-2.0 * log(unit_uniform(x.x))), ta = 2.0 * M_PI * unit_uniform(x.y);
  const double rb = sqrt(-2.0 * log(unit_uniform(x.z))), tb = 2.0 * M_PI * unit_uniform(x.w);
  double z[4];
  sincos(ta, &z[1], &z[0]);
  sincos(tb, &z[3], &z[2]);
  z[0] *= ra;
  z[1] *= ra;
  z[2] *= rb;
  z[3] *= rb;
  for (int m = 0; m < 4; ++m) {
    const int q = 4 * blk + m;
    if (q < N3) r_prop[b * N3 + q] = r[b * N3 + q] + (T)(step * z[m]);
  }
}

// One launch over several molecules: block b runs entry m of the table.
template <class T>
__global__ void propose_kernel_group(const __grid_constant__ Grp<propose_kernel_args<T>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  GRP_STATIC(m_, const auto& a_ = g.a[K_];
             propose_kernel_body<T>(grp_bx(g, K_, l_), grp_by(g, K_, l_), g.nbx[K_], a_.r, a_.r_prop, a_.B, a_.N3, a_.step, a_.seed, a_.t, a_.t_base);)
}

template <class T>
struct accept_kernel_args {
  T* r;
  T* logabs;
  const T* r_prop;
  const T* la_prop;
  const int8_t* sign_prop;
  int64_t B;
  int N3;
  uint64_t seed;
  uint64_t t;
  const uint64_t* t_base;
  unsigned long long* n_acc;
  T* e_loc;            // nullable: local energies carried with the positions
  const T* e_prop;     // the proposals' local energies (with e_loc)
};

template <class T>
__device__ __forceinline__ void accept_kernel_body(const int64_t bx_, const int by_, const int64_t nbx_, T* __restrict__ r, T* __restrict__ logabs, const T* __restrict__ r_prop,
                              const T* __restrict__ la_prop, const int8_t* __restrict__ sign_prop, int64_t B, int N3,
                              uint64_t seed, uint64_t t, const uint64_t* __restrict__ t_base,
                              unsigned long long* __restrict__ n_acc, T* __restrict__ e_loc,
                              const T* __restrict__ e_prop) {
  if (t_base) t += *t_base;
  const int64_t b = (int64_t)bx_ * blockDim.x + threadIdx.x;
  bool acc = false;
  if (b < B) {
    const uint4 ctr = make_uint4((uint32_t)b, (uint32_t)t, kTagAccept << 24, (uint32_t)(t >> 32));
    const uint4 x = philox4x32_10(ctr, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const double lu = log(unit_uniform(x.x));
    acc = sign_prop[b] != 0 && lu < 2.0 * ((double)la_prop[b] - (double)logabs[b]);
    if (acc) {
      for (int q = 0; q < N3; ++q) r[b * N3 + q] = r_prop[b * N3 + q];
      logabs[b] = la_prop[b];
      if (e_loc) e_loc[b] = e_prop[b];
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, acc);
  if ((threadIdx.x % 32) == 0 && m && n_acc) atomicAdd(n_acc, (unsigned long long)__popc(m));
}

// One launch over several molecules: block b runs entry m of the table.
template <class T>
__global__ void accept_kernel_group(const __grid_constant__ Grp<accept_kernel_args<T>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  GRP_STATIC(m_, const auto& a_ = g.a[K_];
             accept_kernel_body<T>(grp_bx(g, K_, l_), grp_by(g, K_, l_), g.nbx[K_], a_.r, a_.logabs, a_.r_prop, a_.la_prop, a_.sign_prop, a_.B, a_.N3, a_.seed, a_.t, a_.t_base, a_.n_acc, a_.e_loc, a_.e_prop);)
}

// ---------------------------------------------------------------------------
// Metropolis-adjusted Langevin step (Sec. 5, the Langevin sampler).  Drift
// v_i = d log|psi| / d r_i per electron, limited as
//   vbar_i = v_i (sqrt(1 + 2 tau |v_i|^2) - 1) / (tau |v_i|^2)
// (Umrigar, Nightingale, Runge 1993, a = 1); proposal r' = r + tau vbar(r) +
// sqrt(tau) xi with the Metropolis sampler's normals; acceptance of
//   log alpha = 2 (log|psi'| - log|psi|) + |xi|^2 / 2 - |r - r' - tau vbar(r')|^2 / (2 tau)
// against the same uniforms (FP64 arithmetic).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ double drift_factor(const T* g, double tau) {  // vbar_i / v_i for the electron at g
  const double v2 = (double)g[0] * g[0] + (double)g[1] * g[1] + (double)g[2] * g[2];
  const double s = tau * v2;
  return s > 0 ? (sqrt(1.0 + 2.0 * s) - 1.0) / s : 1.0;
}

template <class T>
__global__ void mala_propose_kernel(const T* __restrict__ r, const T* __restrict__ g, T* __restrict__ r_prop,
                                    T* __restrict__ xi_out, int64_t B, int N3, double tau, uint64_t seed, uint64_t t,
                                    const uint64_t* __restrict__ t_base) {
  if (t_base) t += *t_base;
  const int nblk = (N3 + 3) / 4;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= B * nblk) return;
  const int64_t b = gid / nblk;
  const int blk = (int)(gid % nblk);
  const uint4 ctr = make_uint4((uint32_t)b, (uint32_t)t, (kTagPropose << 24) | (uint32_t)blk, (uint32_t)(t >> 32));
  const uint4 x = philox4x32_10(ctr, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const double ra = sqrt(-2.0 * log(unit_uniform(x.x))), ta = 2.0 * M_PI * unit_uniform(x.y);
  const double rb = sqrt(-2.0 * log(unit_uniform(x.z))), tb = 2.0 * M_PI * unit_uniform(x.w);
  double z[4];
  sincos(ta, &z[1], &z[0]);
  sincos(tb, &z[3], &z[2]);
  z[0] *= ra;
  z[1] *= ra;
  z[2] *= rb;
  z[3] *= rb;
  const double sq = sqrt(tau);
  for (int m = 0; m < 4; ++m) {
    const int q = 4 * blk + m;
    if (q >= N3) break;
    const T* gi = g + b * N3 + (q / 3) * 3;
    const double vbar = drift_factor(gi, tau) * (double)g[b * N3 + q];
    r_prop[b * N3 + q] = (T)((double)r[b * N3 + q] + tau * vbar + sq * z[m]);
    xi_out[b * N3 + q] = (T)z[m];
  }
}

template <class T>
__global__ void mala_accept_kernel(T* __restrict__ r, T* __restrict__ logabs, T* __restrict__ g,
                                   const T* __restrict__ r_prop, const T* __restrict__ la_prop,
                                   const int8_t* __restrict__ sign_prop, const T* __restrict__ g_prop,
                                   const T* __restrict__ xi, T* __restrict__ e_loc, const T* __restrict__ e_prop,
                                   int64_t B, int N3, double tau, uint64_t seed, uint64_t t,
                                   const uint64_t* __restrict__ t_base, unsigned long long* __restrict__ n_acc) {
  if (t_base) t += *t_base;
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool acc = false;
  if (b < B) {
    const T* rb = r + b * N3;
    const T* rp = r_prop + b * N3;
    const T* gp = g_prop + b * N3;
    double fwd = 0.0, bwd = 0.0;
    for (int q = 0; q < N3; q += 3) {
      const double f = drift_factor(gp + q, tau);
      for (int x = 0; x < 3; ++x) {
        const double z = (double)xi[b * N3 + q + x];
        fwd += z * z;
        const double e = (double)rb[q + x] - (double)rp[q + x] - tau * f * (double)gp[q + x];
        bwd += e * e;
      }
    }
    const uint4 ctr = make_uint4((uint32_t)b, (uint32_t)t, kTagAccept << 24, (uint32_t)(t >> 32));
    const uint4 x = philox4x32_10(ctr, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const double lu = log(unit_uniform(x.x));
    const double la = 2.0 * ((double)la_prop[b] - (double)logabs[b]) + 0.5 * fwd - bwd / (2.0 * tau);
    acc = sign_prop[b] != 0 && lu < la;
    if (acc) {
      for (int q = 0; q < N3; ++q) {
        r[b * N3 + q] = rp[q];
        g[b * N3 + q] = gp[q];
      }
      logabs[b] = la_prop[b];
      if (e_loc) e_loc[b] = e_prop[b];
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, acc);
  if ((threadIdx.x % 32) == 0 && m && n_acc) atomicAdd(n_acc, (unsigned long long)__popc(m));
}

// Deterministic FP64 sums of the finite local energies: one CTA, fixed order.
constexpr int kRedThreads = 1024;

template <class T>
struct esum_kernel_args {
  const T* e;
  int64_t B;
  double* out2;
  unsigned int* status;
};

template <class T>
__device__ __forceinline__ void esum_kernel_body(const int64_t bx_, const int by_, const int64_t nbx_, const T* __restrict__ e, int64_t B, double* __restrict__ out2, unsigned int* status) {
  __shared__ double s1[kRedThreads], s2[kRedThreads];
  double a = 0, q = 0;
  bool bad = false;
  for (int64_t i = threadIdx.x; i < B; i += kRedThreads) {
    const double v = (double)e[i];
    if (isfinite(v)) {
      a += v;
      q += v * v;
    } else {
      bad = true;
    }
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = q;
  if (bad) atomicOr(status, (unsigned)DQ_FLAG_NONFINITE);
  __syncthreads();
  for (int o = kRedThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out2[0] = s1[0];
    out2[1] = s2[0];
  }
}

// One launch over several molecules: block b runs entry m of the table.
template <class T>
__global__ void __launch_bounds__(kRedThreads) esum_kernel_group(const __grid_constant__ Grp<esum_kernel_args<T>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  GRP_STATIC(m_, const auto& a_ = g.a[K_];
             esum_kernel_body<T>(grp_bx(g, K_, l_), grp_by(g, K_, l_), g.nbx[K_], a_.e, a_.B, a_.out2, a_.status);)
}

__device__ double block_sum_det(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = kRedThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Median / mean-absolute-deviation clipping and gradient weights (Sec. 4.4).
// One CTA: bitonic sort of a padded FP64 copy in global scratch, then
// block reductions in a fixed order.
template <class T>
struct loss_weights_kernel_args {
  const T* e;
  int64_t B;
  int64_t Bp;
  double k;
  int soft;
  T* w;
  double* stats;
  double* srt;
};

// Clipped energy: the clamp to [lo, hi], or (soft) the identity inside
// |v - mu| <= sigma and mu + sign(v - mu) sigma (1 + ln(|v - mu| / sigma))
// outside, the logarithmically growing window of Sec. 4.4.
__device__ __forceinline__ double clip_energy(double v, double med, double sig, double lo, double hi, int soft) {
  if (!soft) return fmin(fmax(v, lo), hi);
  const double u = v - med, a = fabs(u);
  if (!(a > sig)) return v;
  return med + copysign(sig * (1.0 + log(a / sig)), u);
}

template <class T>
__device__ __forceinline__ void loss_weights_kernel_body(const int64_t bx_, const int by_, const int64_t nbx_, const T* __restrict__ e, int64_t B, int64_t Bp, double k, int soft, T* __restrict__ w,
                        double* __restrict__ stats, double* __restrict__ srt) {
  __shared__ double sh[kRedThreads];
  for (int64_t i = threadIdx.x; i < Bp; i += kRedThreads) srt[i] = i < B ? (double)e[i] : INFINITY;
  __syncthreads();
  for (int64_t size = 2; size <= Bp; size <<= 1) {
    for (int64_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (int64_t i = threadIdx.x; i < Bp; i += kRedThreads) {
        const int64_t j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const double a = srt[i], c = srt[j];
          if ((a > c) == up) {
            srt[i] = c;
            srt[j] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  const double med = (B % 2) ? srt[B / 2] : 0.5 * (srt[B / 2 - 1] + srt[B / 2]);
  double part = 0, raw = 0;
  for (int64_t i = threadIdx.x; i < B; i += kRedThreads) {
    const double v = (double)e[i];
    part += fabs(v - med);
    raw += v;
  }
  const double mad = block_sum_det(part, sh) / (double)B;
  const double mean_raw = block_sum_det(raw, sh) / (double)B;
  const double sig = k * mad, lo = med - sig, hi = med + sig;
  double cs = 0;
  for (int64_t i = threadIdx.x; i < B; i += kRedThreads) cs += clip_energy((double)e[i], med, sig, lo, hi, soft);
  const double mean_c = block_sum_det(cs, sh) / (double)B;
  for (int64_t i = threadIdx.x; i < B; i += kRedThreads)
    w[i] = (T)((2.0 / (double)B) * (clip_energy((double)e[i], med, sig, lo, hi, soft) - mean_c));
  if (threadIdx.x == 0 && stats) {
    stats[0] = med;
    stats[1] = k * mad;
    stats[2] = mean_c;
    stats[3] = mean_raw;
  }
}

// One launch over several molecules: block b runs entry m of the table.
template <class T>
__global__ void __launch_bounds__(kRedThreads) loss_weights_kernel_group(const __grid_constant__ Grp<loss_weights_kernel_args<T>> g) {
  int64_t l_;
  const int m_ = grp_find(g, blockIdx.x, l_);
  GRP_STATIC(m_, const auto& a_ = g.a[K_];
             loss_weights_kernel_body<T>(grp_bx(g, K_, l_), grp_by(g, K_, l_), g.nbx[K_], a_.e, a_.B, a_.Bp, a_.k, a_.soft, a_.w, a_.stats, a_.srt);)
}

}  // namespace

__global__ void advance_counter_kernel(uint64_t* c, uint64_t n) { *c += n; }

// Single-molecule launchers: the grouped kernels with a one-entry table.
template <class T>
cudaError_t launch_propose(const dq_handle_s& h, int64_t B, const T* r, T* r_prop, double step, uint64_t seed,
                           uint64_t t, const uint64_t* t_base, cudaStream_t s) {
  const dq_handle_s* hp = &h;
  return launch_propose_group<T>(&hp, 1, &B, &r, &r_prop, step, seed, t, t_base, s);
}

template <class T>
cudaError_t launch_mala_propose(const dq_handle_s& h, int64_t B, const T* r, const T* g, T* r_prop, T* xi,
                                double tau, uint64_t seed, uint64_t t, const uint64_t* t_base, cudaStream_t s) {
  const int N3 = 3 * h.N, nblk = (N3 + 3) / 4;
  const int64_t n = B * nblk;
  mala_propose_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(r, g, r_prop, xi, B, N3, tau, seed, t, t_base);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_mala_accept(const dq_handle_s& h, int64_t B, T* r, T* logabs, T* g, const T* r_prop,
                               const T* la_prop, const int8_t* sign_prop, const T* g_prop, const T* xi, T* e_loc,
                               const T* e_prop, double tau, uint64_t seed, uint64_t t, const uint64_t* t_base,
                               unsigned long long* n_acc, cudaStream_t s) {
  mala_accept_kernel<T><<<(unsigned)((B + 255) / 256), 256, 0, s>>>(
      r, logabs, g, r_prop, la_prop, sign_prop, g_prop, xi, e_loc, e_prop, B, 3 * h.N, tau, seed, t, t_base, n_acc);
  return cudaGetLastError();
}

cudaError_t launch_advance_counter(uint64_t* c, uint64_t n, cudaStream_t s) {
  advance_counter_kernel<<<1, 1, 0, s>>>(c, n);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_accept(const dq_handle_s& h, int64_t B, T* r, T* logabs, const T* r_prop, const T* logabs_prop,
                          const int8_t* sign_prop, uint64_t seed, uint64_t t, const uint64_t* t_base,
                          unsigned long long* n_acc, cudaStream_t s, T* e_loc, const T* e_prop) {
  const dq_handle_s* hp = &h;
  return launch_accept_group<T>(&hp, 1, &B, &r, &logabs, &r_prop, &logabs_prop, &sign_prop, seed, t, t_base, &n_acc,
                                s, e_loc, e_prop);
}

template <class T>
cudaError_t launch_esum(const T* e, int64_t B, double* out2, unsigned int* status, cudaStream_t s) {
  return launch_esum_group<T>(1, &e, &B, &out2, &status, s);
}

template <class T>
cudaError_t launch_loss_weights(const T* e, int64_t B, double k, T* w, double* stats, double* scratch,
                                cudaStream_t s, int soft) {
  return launch_loss_weights_group<T>(1, &e, &B, k, &w, stats ? &stats : nullptr, &scratch, s, soft);
}

// Grouped launches: one launch per sampler step over every molecule of a batch
// (entry m: molecule m's walkers, buffers and accept counter).  Molecule m's
// draws are those of the single-molecule calls with the same seed and step.
template <class T>
cudaError_t launch_propose_group(const dq_handle_s* const* hs, int n, const int64_t* B, const T* const* r,
                                 T* const* r_prop, double step, uint64_t seed, uint64_t t, const uint64_t* t_base,
                                 cudaStream_t s) {
  if (n > kMaxGroup) return cudaErrorInvalidValue;
  Grp<propose_kernel_args<T>> g{};
  for (int k = 0; k < n; ++k) {
    if (B[k] <= 0) continue;
    const int N3 = 3 * hs[k]->N, nblk = (N3 + 3) / 4;
    g.add({r[k], r_prop[k], B[k], N3, step, seed, t, t_base}, (B[k] * nblk + 255) / 256);
  }
  if (g.n == 0) return cudaSuccess;
  propose_kernel_group<T><<<(unsigned)g.blocks(), 256, 0, s>>>(g);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_accept_group(const dq_handle_s* const* hs, int n, const int64_t* B, T* const* r, T* const* logabs,
                                const T* const* r_prop, const T* const* la_prop, const int8_t* const* sign_prop,
                                uint64_t seed, uint64_t t, const uint64_t* t_base, unsigned long long* const* n_acc,
                                cudaStream_t s, T* e_loc, const T* e_prop) {
  if (n > kMaxGroup) return cudaErrorInvalidValue;
  Grp<accept_kernel_args<T>> g{};
  for (int k = 0; k < n; ++k) {
    if (B[k] <= 0) continue;
    g.add({r[k], logabs[k], r_prop[k], la_prop[k], sign_prop[k], B[k], 3 * hs[k]->N, seed, t, t_base,
           n_acc ? n_acc[k] : nullptr, n == 1 ? e_loc : nullptr, n == 1 ? e_prop : nullptr},
          (B[k] + 255) / 256);
  }
  if (g.n == 0) return cudaSuccess;
  accept_kernel_group<T><<<(unsigned)g.blocks(), 256, 0, s>>>(g);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_esum_group(int n, const T* const* e, const int64_t* B, double* const* out2,
                              unsigned int* const* status, cudaStream_t s) {
  if (n > kMaxGroup) return cudaErrorInvalidValue;
  Grp<esum_kernel_args<T>> g{};
  for (int k = 0; k < n; ++k)
    if (out2[k]) g.add({e[k], B[k], out2[k], status[k]}, 1);
  if (g.n == 0) return cudaSuccess;
  esum_kernel_group<T><<<(unsigned)g.blocks(), kRedThreads, 0, s>>>(g);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_loss_weights_group(int n, const T* const* e, const int64_t* B, double k, T* const* w,
                                      double* const* stats, double* const* scratch, cudaStream_t s, int soft) {
  if (n > kMaxGroup) return cudaErrorInvalidValue;
  Grp<loss_weights_kernel_args<T>> g{};
  for (int m = 0; m < n; ++m) {
    if (B[m] <= 0) continue;
    int64_t Bp = 1;
    while (Bp < B[m]) Bp <<= 1;
    g.add({e[m], B[m], Bp, k, soft, w[m], stats ? stats[m] : nullptr, scratch[m]}, 1);
  }
  if (g.n == 0) return cudaSuccess;
  loss_weights_kernel_group<T><<<(unsigned)g.blocks(), kRedThreads, 0, s>>>(g);
  return cudaGetLastError();
}

#define DQ_INST_GROUP(T)                                                                                           \
  template cudaError_t launch_propose_group<T>(const dq_handle_s* const*, int, const int64_t*, const T* const*,     \
                                               T* const*, double, uint64_t, uint64_t, const uint64_t*,            \
                                               cudaStream_t);                                                     \
  template cudaError_t launch_accept_group<T>(const dq_handle_s* const*, int, const int64_t*, T* const*, T* const*, \
                                              const T* const*, const T* const*, const int8_t* const*, uint64_t,   \
                                              uint64_t, const uint64_t*, unsigned long long* const*,             \
                                              cudaStream_t, T*, const T*);                                        \
  template cudaError_t launch_esum_group<T>(int, const T* const*, const int64_t*, double* const*,                  \
                                            unsigned int* const*, cudaStream_t);                                  \
  template cudaError_t launch_loss_weights_group<T>(int, const T* const*, const int64_t*, double, T* const*,       \
                                                    double* const*, double* const*, cudaStream_t, int);
DQ_INST_GROUP(float)
DQ_INST_GROUP(double)

#define DQ_INST(T)                                                                                                 \
  template cudaError_t launch_propose<T>(const dq_handle_s&, int64_t, const T*, T*, double, uint64_t, uint64_t,    \
                                         const uint64_t*, cudaStream_t);                                          \
  template cudaError_t launch_accept<T>(const dq_handle_s&, int64_t, T*, T*, const T*, const T*, const int8_t*,    \
                                        uint64_t, uint64_t, const uint64_t*, unsigned long long*, cudaStream_t,   \
                                        T*, const T*);                                                            \
  template cudaError_t launch_mala_propose<T>(const dq_handle_s&, int64_t, const T*, const T*, T*, T*, double,      \
                                              uint64_t, uint64_t, const uint64_t*, cudaStream_t);                 \
  template cudaError_t launch_mala_accept<T>(const dq_handle_s&, int64_t, T*, T*, T*, const T*, const T*,          \
                                             const int8_t*, const T*, const T*, T*, const T*, double, uint64_t,   \
                                             uint64_t,                                                            \
                                             const uint64_t*, unsigned long long*, cudaStream_t);                 \
  template cudaError_t launch_esum<T>(const T*, int64_t, double*, unsigned int*, cudaStream_t);                   \
  template cudaError_t launch_loss_weights<T>(const T*, int64_t, double, T*, double*, double*, cudaStream_t, int);
DQ_INST(float)
DQ_INST(double)

}  // namespace dq
