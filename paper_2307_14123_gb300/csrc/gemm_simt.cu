// Plain FP32 / FP64 GEMM on CUDA cores for the jet-propagating linear layers.
//
//   Y[r][n] (+)= sum_k X[r][k] W[n][k] + bias[n]   (bias on rows r % period == 0)
//
// Rows of X and Y are addressed through a segmented row map so that one launch
// covers, e.g., all walkers' spin-up rows of the orbital head, or all
// same-spin edges of a chunk.  In the jet layout a row is one channel (value,
// one of the 3N first derivatives, or the Laplacian) of one node; a linear map
// acts on every channel alike and the bias only on the value channel, which is
// how value, Jacobian and Laplacian propagate through Eqs. (17)-(19), (24).
//
// Tiling: BM x BN output tile per CTA, BK-deep k-slices double-buffered in
// shared memory (transposed, padded, 16-byte vector accesses), TM x TN
// register tile per thread split in two halves so that shared-memory reads
// are conflict-free.
#include "common.cuh"

namespace dq {
namespace {

template <class T>
struct Vec;
template <>
struct Vec<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec<double> {
  using type = double2;
  static constexpr int n = 2;
};

__device__ __forceinline__ int64_t row_offset(const RowMap& m, int64_t r) {
  return (r / m.rows_per_seg) * m.seg_stride + (r % m.rows_per_seg) * m.ld;
}

// XA / WA: rows of X / W start on 16-byte boundaries (vector loads), else
// VEC scalar loads are used (parameter blocks of the flat vector need not be
// aligned).
template <class T, int BM, int BN, int BK, bool XA, bool WA>
__global__ void __launch_bounds__(256)
    gemm_nt_kernel(const T* __restrict__ X, RowMap mx, const T* __restrict__ W, const T* __restrict__ bias,
                   int bias_period, T* __restrict__ Y, RowMap my, int64_t rows, int n_out, int K, int accumulate) {
  using V = typename Vec<T>::type;
  constexpr int VEC = Vec<T>::n;
  constexpr int NT = 256;
  constexpr int TM = 2 * VEC, TN = 2 * VEC;
  static_assert((BM / TM) * (BN / TN) == NT, "tile/thread mismatch");
  constexpr int KV = BK / VEC;
  constexpr int LA = BM * KV / NT;
  constexpr int LB = BN * KV / NT;
  static_assert(LA >= 1 && LB >= 1 && BM * KV % NT == 0 && BN * KV % NT == 0, "load split");
  constexpr int PAD = VEC;
  __shared__ __align__(16) T As[2][BK][BM + PAD];
  __shared__ __align__(16) T Bs[2][BK][BN + PAD];

  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int col0 = blockIdx.y * BN;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);

  const T* a_ptr[LA];
  int a_row[LA], a_kv[LA];
  bool a_ok[LA];
#pragma unroll
  for (int i = 0; i < LA; ++i) {
    const int l = tid + i * NT;
    a_row[i] = l / KV;
    a_kv[i] = l % KV;
    const int64_t r = row0 + a_row[i];
    a_ok[i] = r < rows;
    a_ptr[i] = X + (a_ok[i] ? row_offset(mx, r) : 0) + a_kv[i] * VEC;
  }
  const T* b_ptr[LB];
  int b_row[LB], b_kv[LB];
  bool b_ok[LB];
#pragma unroll
  for (int i = 0; i < LB; ++i) {
    const int l = tid + i * NT;
    b_row[i] = l / KV;
    b_kv[i] = l % KV;
    const int n = col0 + b_row[i];
    b_ok[i] = n < n_out;
    b_ptr[i] = W + (b_ok[i] ? (int64_t)n * K : 0) + b_kv[i] * VEC;
  }

  V ra[LA], rb[LB];
  auto load = [&](int k0) {
#pragma unroll
    for (int i = 0; i < LA; ++i) {
      if (a_ok[i]) {
        if constexpr (XA) {
          ra[i] = *reinterpret_cast<const V*>(a_ptr[i] + k0);
        } else {
          T* v = reinterpret_cast<T*>(&ra[i]);
#pragma unroll
          for (int e = 0; e < VEC; ++e) v[e] = a_ptr[i][k0 + e];
        }
      } else {
        ra[i] = V{};
      }
    }
#pragma unroll
    for (int i = 0; i < LB; ++i) {
      if (b_ok[i]) {
        if constexpr (WA) {
          rb[i] = __ldg(reinterpret_cast<const V*>(b_ptr[i] + k0));
        } else {
          T* v = reinterpret_cast<T*>(&rb[i]);
#pragma unroll
          for (int e = 0; e < VEC; ++e) v[e] = __ldg(b_ptr[i] + k0 + e);
        }
      } else {
        rb[i] = V{};
      }
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < LA; ++i) {
      const T* v = reinterpret_cast<const T*>(&ra[i]);
#pragma unroll
      for (int e = 0; e < VEC; ++e) As[buf][a_kv[i] * VEC + e][a_row[i]] = v[e];
    }
#pragma unroll
    for (int i = 0; i < LB; ++i) {
      const T* v = reinterpret_cast<const T*>(&rb[i]);
#pragma unroll
      for (int e = 0; e < VEC; ++e) Bs[buf][b_kv[i] * VEC + e][b_row[i]] = v[e];
    }
  };

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  load(0);
  store(0);
  __syncthreads();
  const int ntiles = K / BK;
  for (int t = 0; t < ntiles; ++t) {
    const int cur = t & 1;
    if (t + 1 < ntiles) load((t + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
      *reinterpret_cast<V*>(&a[0]) = *reinterpret_cast<const V*>(&As[cur][kk][ty * VEC]);
      *reinterpret_cast<V*>(&a[VEC]) = *reinterpret_cast<const V*>(&As[cur][kk][BM / 2 + ty * VEC]);
      *reinterpret_cast<V*>(&b[0]) = *reinterpret_cast<const V*>(&Bs[cur][kk][tx * VEC]);
      *reinterpret_cast<V*>(&b[VEC]) = *reinterpret_cast<const V*>(&Bs[cur][kk][BN / 2 + tx * VEC]);
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (t + 1 < ntiles) store(cur ^ 1);
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int lr = (i < VEC) ? ty * VEC + i : BM / 2 + ty * VEC + (i - VEC);
    const int64_t r = row0 + lr;
    if (r >= rows) continue;
    T* y = Y + row_offset(my, r);
    const bool add_bias = bias != nullptr && (r % bias_period) == 0;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int lc = (j < VEC) ? tx * VEC + j : BN / 2 + tx * VEC + (j - VEC);
      const int n = col0 + lc;
      if (n >= n_out) continue;
      T v = acc[i][j];
      if (add_bias) v += bias[n];
      if (accumulate) v += y[n];
      y[n] = v;
    }
  }
}

}  // namespace

namespace {
template <class T, int BM, int BN, int BK>
cudaError_t gemm_dispatch(const T* X, RowMap mx, const T* W, const T* bias, int bias_period, T* Y, RowMap my,
                          int64_t rows, int n_out, int K, bool accumulate, cudaStream_t s) {
  constexpr int VEC = Vec<T>::n;
  const bool xa = (uintptr_t)X % 16 == 0 && mx.ld % VEC == 0 && mx.seg_stride % VEC == 0;
  const bool wa = (uintptr_t)W % 16 == 0;
  dim3 grid((unsigned)((rows + BM - 1) / BM), (unsigned)((n_out + BN - 1) / BN));
  const int acc = accumulate ? 1 : 0;
  if (xa && wa)
    gemm_nt_kernel<T, BM, BN, BK, true, true><<<grid, 256, 0, s>>>(X, mx, W, bias, bias_period, Y, my, rows, n_out, K, acc);
  else if (xa)
    gemm_nt_kernel<T, BM, BN, BK, true, false><<<grid, 256, 0, s>>>(X, mx, W, bias, bias_period, Y, my, rows, n_out, K, acc);
  else if (wa)
    gemm_nt_kernel<T, BM, BN, BK, false, true><<<grid, 256, 0, s>>>(X, mx, W, bias, bias_period, Y, my, rows, n_out, K, acc);
  else
    gemm_nt_kernel<T, BM, BN, BK, false, false><<<grid, 256, 0, s>>>(X, mx, W, bias, bias_period, Y, my, rows, n_out, K, acc);
  return cudaGetLastError();
}
}  // namespace

template <class T>
cudaError_t gemm_nt(const T* X, RowMap mx, const T* W, const T* bias, int bias_period, T* Y, RowMap my,
                    int64_t rows, int n_out, int K, bool accumulate, cudaStream_t s) {
  if (rows <= 0 || n_out <= 0) return cudaSuccess;
  if (K % 8 != 0 || bias_period <= 0) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 4) {
    return gemm_dispatch<T, 128, 128, 8>(X, mx, W, bias, bias_period, Y, my, rows, n_out, K, accumulate, s);
  } else {
    return gemm_dispatch<T, 64, 64, 8>(X, mx, W, bias, bias_period, Y, my, rows, n_out, K, accumulate, s);
  }
}

template cudaError_t gemm_nt<float>(const float*, RowMap, const float*, const float*, int, float*, RowMap,
                                    int64_t, int, int, bool, cudaStream_t);
template cudaError_t gemm_nt<double>(const double*, RowMap, const double*, const double*, int, double*,
                                     RowMap, int64_t, int, int, bool, cudaStream_t);

}  // namespace dq
