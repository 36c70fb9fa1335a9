// Warp-level dense linear algebra on small matrices in shared memory, used by
// the determinant kernels (forward and reverse): LU with partial pivoting (the
// pivot search is a warp-wide argmax), log|det| and sign, and the inverse.
#pragma once

#include <math.h>

namespace dq {
namespace {

template <class S>
__device__ __forceinline__ S warp_max(S v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// In-place LU with partial pivoting of the n x n matrix LU (row-major, shared
// memory) by one warp; perm records the row order.  Returns false if a zero
// pivot appears.  sign and logabs of the determinant are accumulated.
template <class S>
__device__ bool warp_lu(S* LU, int* perm, int n, int lane, int* sign_out, double* logabs_out) {
  if (lane < n) perm[lane] = lane;
  __syncwarp();
  int sign = 1;
  S la = 0;
  for (int j = 0; j < n; ++j) {
    S v = (lane >= j && lane < n) ? fabs(LU[lane * n + j]) : S(-1);
    int idx = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const S v2 = __shfl_xor_sync(0xffffffffu, v, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
      if (v2 > v || (v2 == v && i2 < idx)) {
        v = v2;
        idx = i2;
      }
    }
    if (!(v > S(0))) return false;
    if (idx != j) {
      for (int k = lane; k < n; k += 32) {
        const S t = LU[j * n + k];
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
    const S piv = LU[j * n + j];
    for (int i = j + 1 + lane; i < n; i += 32) {
      const S f = LU[i * n + j] / piv;
      LU[i * n + j] = f;
      for (int k = j + 1; k < n; ++k) LU[i * n + k] -= f * LU[j * n + k];
    }
    __syncwarp();
    if (piv < S(0)) sign = -sign;
    if (lane == (j & 31)) la += log(fabs(piv));  // one lane per pivot, summed below
  }
  *sign_out = sign;
  double l = (double)la;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  *logabs_out = l;
  return true;
}

// A^-1 from the LU factors: lane `col` solves L U x = P e_col.
template <class S>
__device__ void warp_inverse(const S* LU, const int* perm, int n, int lane, S* Ainv) {
  if (lane < n) {
    const int col = lane;
    for (int r = 0; r < n; ++r) {
      S acc = perm[r] == col ? S(1) : S(0);
      for (int m = 0; m < r; ++m) acc -= LU[r * n + m] * Ainv[m * n + col];
      Ainv[r * n + col] = acc;
    }
    for (int r = n - 1; r >= 0; --r) {
      S acc = Ainv[r * n + col];
      for (int m = r + 1; m < n; ++m) acc -= LU[r * n + m] * Ainv[m * n + col];
      Ainv[r * n + col] = acc / LU[r * n + r];
    }
  }
  __syncwarp();
}

// Double-float arithmetic (an FP32 pair hi + lo) from error-free
// transformations: TwoSum (Knuth) and TwoProd via a fused multiply-add
// (Ogita, Rump, Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput.
// 26, 2005).  Explicit round-to-nearest intrinsics keep the compiler from
// contracting the operations that must stay exact.
struct dfloat {
  float hi, lo;
};
__device__ __forceinline__ dfloat two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dfloat quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  dfloat s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return quick_two_sum(p, e);
}
// sum_l a[l] b[l] as a double-float pair (Dot2)
__device__ __forceinline__ dfloat dot2_step(dfloat acc, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const dfloat s = two_sum(acc.hi, p);
  return {s.hi, __fadd_rn(acc.lo, __fadd_rn(s.lo, e))};
}

__device__ __forceinline__ dfloat warp_sum_df(dfloat v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dfloat w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = df_add(v, w);
  }
  return v;
}

}  // namespace
}  // namespace dq
