// Jet messages of Eq. 17 for molecules beyond the fused layer kernel (FP32 modes, node
// channels from the node map): for every receiver i, channel c and feature,
//   m_i^t[c] = nu_t ( sum_{j in block t} w_ij z_j[c] + product-rule terms ),
// the product-rule terms being those listed with the general message kernel in forward.cu:
//  (a) a sender's coordinate channel c = 1 + 3e + x:  -w'_ie u_ie,x z_e[0];
//  (b) the receiver's own coordinate channel:         sum_j w'_ij u_ij,x z_j[0];
//  (c) the Laplacian channel: sum_j (2 w''_ij + 4 w'_ij / d_ij) z_j[0] + 2 w'_ij u_ij.(dz_j/dr_i - dz_j/dr_j);
//  and the electron-nucleus messages, non-zero on the value, Laplacian and own-coordinate
//  channels only.
//
// One CTA per (walker, 32 features), a lane per feature, 16 warps.  The senders are taken one
// spin block at a time: pass p holds the senders of block p, which give a receiver of block p its
// same-spin message and every other receiver its opposite-spin one.  Per pass, w_ij, w'_ij and
// w''_ij of the block's senders and all receivers are copied into shared memory as [j][i][32]
// (16-byte asynchronous copies; rows past the block and the diagonal are zero).  A warp task
// owns the 3 EPT coordinate channels of EPT consecutive electrons (one more task the value and
// Laplacian channels): it loads z_j[c] of the block's NBS sender slots for them into registers
// (each value of z is read by exactly one task, coalesced over the features) and runs over all
// receivers, NBS x 3 EPT multiply-adds per receiver against NBS conflict-free shared-memory
// loads of w; with the channels aligned to electrons, the product-rule terms of a register slot
// have a fixed electron and axis and are added without branches before the store.  The task
// also forms the pass's sums (b) and (c) for its electrons as receivers, the cross term of (c)
// from the dz_j / dr_e it holds; the Laplacian channel is completed after all tasks.
//
// The general kernel (forward.cu) streams the senders' node channels four senders at a time
// through 4-byte copies per lane, with the w tables of all N^2 pairs resident; here z lives in
// registers, read once, and only one spin block's tables are resident (at 28 electrons this
// kernel takes half the general kernel's time).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace dq {
namespace {

constexpr int kMLLanes = 32;   // features per CTA
constexpr int kMLMaxN = 48;    // electrons

struct MLArgs {
  const float* Z;      // [Bc][N][C][D] node map z_j
  const float* ew;     // [Bc][E][3][D] filter jets w, dw/dd, d2w/dd2
  const float* geo;    // [Bc][E][4] distance and unit vector of every edge
  const float* Y;      // [M][D] nucleus embeddings of the layer
  const int* pair_of;  // [N][N] edge of (i, j), -1 on the diagonal
  void* msg;           // [Bc][N][C][3D] messages [same spin | opposite spin | nuclei]
  int N, n_up, M, C, D, E, n_ee;
  int stage_w1;        // w' and w'' tables in shared memory (else read from global memory)
};

// Shared-memory layout in floats (the pair table in ints at the same scale).
struct MLSmem {
  int ps, us, id, z0c, zsf, spb, spc, lap, w0, w1, w2, total_bytes;
};
__host__ __device__ inline MLSmem ml_layout(int N, int NBS, bool stage_w1) {
  MLSmem m{};
  int o = 0;
  m.ps = o; o += N * N;
  m.us = o; o += N * N * 3;
  m.id = o; o += N * N;
  m.z0c = o; o += N * kMLLanes;
  m.zsf = o; o += 3 * N * kMLLanes;
  m.spb = o; o += 3 * N * kMLLanes;
  m.spc = o; o += N * kMLLanes;
  m.lap = o; o += N * kMLLanes;
  o = (o + 3) / 4 * 4;  // 16-byte alignment of the copied tables
  m.w0 = o; o += NBS * N * kMLLanes;
  m.w1 = o; o += stage_w1 ? NBS * N * kMLLanes : 0;
  m.w2 = o; o += stage_w1 ? NBS * N * kMLLanes : 0;
  m.total_bytes = o * 4;
  return m;
}

__device__ __forceinline__ void store_out(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_out(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, bool valid) {
  // a zero-sized source fills the 16 bytes with zeros
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

// NBS: sender slots per spin block (at least the larger block); EPT: electrons per warp task (its
// register tile is NBS x 3 EPT); NW: warps per CTA; SW1: the w' tables in shared memory (else read
// from global memory where used).
template <int NBS, int EPT, int NW, bool SW1, class TO>
__global__ void __launch_bounds__(NW * 32, 1) messages_large_kernel(const __grid_constant__ MLArgs a) {
  constexpr int CB = 3 * EPT;
  extern __shared__ __align__(16) float ml_smem[];
  const int N = a.N, C = a.C, D = a.D, M = a.M, n_up = a.n_up, n_ee = a.n_ee;
  const MLSmem lay = ml_layout(N, NBS, SW1);
  int* Ps = reinterpret_cast<int*>(ml_smem + lay.ps);  // [i][j] edge
  float* Us = ml_smem + lay.us;                        // [i][j][3] u_ij (zero diagonal)
  float* Id = ml_smem + lay.id;                        // [i][j] 1 / d_ij
  float* Z0c = ml_smem + lay.z0c;                      // [j][32] z_j[0]
  float* Zsf = ml_smem + lay.zsf;                      // [j][x][32] dz_j / dr_j,x
  float* SPb = ml_smem + lay.spb;                      // [i][x][32] (b) of the pass
  float* SPc = ml_smem + lay.spc;                      // [i][32] (c) of the pass
  float* LAP = ml_smem + lay.lap;                      // [i][32] Laplacian-channel contraction
  float* W0 = ml_smem + lay.w0;                        // [jj][i][32] w of the pass's senders
  float* W1 = ml_smem + lay.w1;                        // [jj][i][32] w'
  float* W2 = ml_smem + lay.w2;                        // [jj][i][32] w''
  constexpr bool stage_w1 = SW1;

  const int64_t b = blockIdx.x;
  const int f0 = blockIdx.y * kMLLanes;
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  const float* EWb = a.ew + b * (int64_t)a.E * 3 * D + f0 + lane;
  const float* Zb = a.Z + b * (int64_t)N * C * D + f0 + lane;
  const float* Yd = a.Y + f0 + lane;
  const float* Gb = a.geo + b * (int64_t)a.E * 4;
  TO* mb = static_cast<TO*>(a.msg) + b * (int64_t)N * C * 3 * D + f0 + lane;
  const int NN = N * N;

  // this CTA's slices of the node channels and filters into L2
  for (int r = tid; r < N * C; r += blockDim.x)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.Z + (b * N * C + r) * (int64_t)D + f0));
  for (int r = tid; r < a.E * 3; r += blockDim.x)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.ew + (b * a.E * 3 + r) * (int64_t)D + f0));

  // ---- per-walker tables ----
  for (int k = tid; k < NN; k += blockDim.x) {
    const int i = k / N, j = k - (k / N) * N;
    const int p = a.pair_of[k];
    Ps[k] = p;
    float u0 = 0.f, u1 = 0.f, u2 = 0.f, id = 0.f;
    if (i != j) {
      const float sg = i < j ? 1.f : -1.f;
      const float4 g = *reinterpret_cast<const float4*>(Gb + p * 4);
      u0 = sg * g.y;
      u1 = sg * g.z;
      u2 = sg * g.w;
      id = 1.f / g.x;
    }
    Us[k * 3] = u0;
    Us[k * 3 + 1] = u1;
    Us[k * 3 + 2] = u2;
    Id[k] = id;
  }
  for (int j = warp; j < N; j += NW) {
    const float* zj = Zb + (int64_t)j * C * D;
    Z0c[j * 32 + lane] = zj[0];
#pragma unroll
    for (int x = 0; x < 3; ++x) Zsf[(j * 3 + x) * 32 + lane] = zj[(int64_t)(1 + 3 * j + x) * D];
  }
  // electron-nucleus slot of receiver i (a warp item): (1/M) sum_I of w_iI Y_I (value channel),
  // w'_iI u_iI,x Y_I (own coordinates), (w''_iI + 2 w'_iI / d_iI) Y_I (Laplacian), zero on the
  // other channels; the loads of eight nuclei are issued before any is used
  const float nuM = 1.f / (float)M;
  for (int i = warp; i < N; i += NW) {
    float sv = 0.f, sx = 0.f, sy = 0.f, sz = 0.f, sl = 0.f;
    for (int I0 = 0; I0 < M; I0 += 8) {
      float w0v[8], w1v[8], w2v[8], yv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool ok = I0 + u < M;
        const int en = n_ee + i * M + (ok ? I0 + u : 0);
        const float* w = EWb + (int64_t)en * 3 * D;
        w0v[u] = ok ? w[0] : 0.f;
        w1v[u] = ok ? w[D] : 0.f;
        w2v[u] = ok ? w[2 * D] : 0.f;
        yv[u] = ok ? Yd[(int64_t)(I0 + u) * D] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (I0 + u >= M) break;
        const float* g = Gb + (n_ee + i * M + I0 + u) * 4;
        sv = fmaf(w0v[u], yv[u], sv);
        sx = fmaf(w1v[u] * g[1], yv[u], sx);
        sy = fmaf(w1v[u] * g[2], yv[u], sy);
        sz = fmaf(w1v[u] * g[3], yv[u], sz);
        sl = fmaf(w2v[u] + 2.f * w1v[u] / g[0], yv[u], sl);
      }
    }
    TO* o = mb + (int64_t)i * C * 3 * D + 2 * D;
    for (int c = 0; c < C; ++c) {
      const float v = c == 0 ? sv : c == C - 1 ? sl : c == 1 + 3 * i ? sx : c == 2 + 3 * i ? sy : c == 3 + 3 * i ? sz : 0.f;
      store_out(o + (int64_t)c * 3 * D, v * nuM);
    }
  }
  __syncthreads();  // pair table, unit vectors, z_j[0]

  const uint32_t w0s = (uint32_t)__cvta_generic_to_shared(W0), w1s = (uint32_t)__cvta_generic_to_shared(W1);
  const uint32_t w2s = (uint32_t)__cvta_generic_to_shared(W2);
  const float* ew_row = a.ew + b * (int64_t)a.E * 3 * D + f0;  // lane-independent row base
  for (int pass = 0; pass < 2; ++pass) {
    const int j0 = pass == 0 ? 0 : n_up, jn = pass == 0 ? n_up : N - n_up;
    // ---- the pass's filter tables: row (jj, i) holds w_{i, j0 + jj} for the 32 features, as
    // eight 16-byte copies (lane / 8 picks one of four rows, lane % 8 the chunk) ----
    {
      const int rows = NBS * N;
      const int sub = lane >> 3, ch = (lane & 7) * 4;
      for (int r0 = warp * 4; r0 < rows; r0 += NW * 4) {
        const int r = r0 + sub;
        if (r < rows) {
          const int jj = r / N, i = r - (r / N) * N;
          const int j = j0 + jj;
          const int p = (jj < jn && i != j) ? Ps[i * N + j] : -1;
          const float* src = ew_row + (int64_t)(p >= 0 ? p : 0) * 3 * D + ch;
          cp16(w0s + (uint32_t)((r * 32 + ch) * 4), src, p >= 0);
          if (stage_w1) {
            cp16(w1s + (uint32_t)((r * 32 + ch) * 4), src + D, p >= 0);
            cp16(w2s + (uint32_t)((r * 32 + ch) * 4), src + 2 * D, p >= 0);
          }
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    auto w1_at = [&](int i, int jj) -> float {  // w'_{i, j0 + jj} of this lane's feature
      if (stage_w1) return W1[(jj * N + i) * 32 + lane];
      const int j = j0 + jj;
      return i == j ? 0.f : EWb[((int64_t)Ps[i * N + j] * 3 + 1) * D];
    };
    // ---- the contraction: a warp task holds the 3 EPT coordinate channels of EPT consecutive
    // electrons (channel c = 1 + 3 e + x: electron e, axis x known per register slot), and one
    // more task the value and Laplacian channels; each runs over all receivers ----
    const float nu_same = 1.f / (float)(jn - 1 > 1 ? jn - 1 : 1), nu_opp = 1.f / (float)(jn > 1 ? jn : 1);
    const int ncoord = (N + EPT - 1) / EPT;
    for (int task = warp; task <= ncoord; task += NW) {
      if (task < ncoord) {
        const int e0 = task * EPT, c0 = 1 + 3 * e0;
        float zr[CB][NBS];
#pragma unroll
        for (int q = 0; q < CB; ++q)
#pragma unroll
          for (int jj = 0; jj < NBS; ++jj)
            zr[q][jj] = (jj < jn && e0 + q / 3 < N) ? Zb[((int64_t)(j0 + jj) * C + c0 + q) * D] : 0.f;
        // (a) per electron slot s: the sender slot of e0 + s and its z_e[0] (zero when e0 + s is not
        // a sender of this pass, which zeroes the term)
        int ja[EPT];
        float za[EPT];
#pragma unroll
        for (int s = 0; s < EPT; ++s) {
          const int e = e0 + s;
          const bool snd = e < N && e >= j0 && e < j0 + jn;
          ja[s] = snd ? e - j0 : 0;
          za[s] = snd ? Z0c[e * 32 + lane] : 0.f;
        }
        // the pass's sums over senders for the task's electrons as receivers: (b) into SPb (read
        // back by this warp only) and (c) into SPc (read by the Laplacian epilogue); the cross term
        // of (c) takes dz_j / dr_e,x from the register tile
#pragma unroll
        for (int s = 0; s < EPT; ++s) {
          const int e = e0 + s;
          if (e >= N) break;
          float b0 = 0.f, b1 = 0.f, b2 = 0.f, sv = 0.f;
          float w2v[SW1 ? 1 : NBS];  // w'' from global memory when the tables are not staged
          if (!SW1) {
#pragma unroll
            for (int jj = 0; jj < NBS; ++jj) {
              const int j = j0 + jj;
              w2v[SW1 ? 0 : jj] = (jj < jn && j != e) ? EWb[((int64_t)Ps[e * N + j] * 3 + 2) * D] : 0.f;
            }
          }
#pragma unroll
          for (int jj = 0; jj < NBS; ++jj) {
            if (jj >= jn) break;
            const int j = j0 + jj;
            const float v1 = w1_at(e, jj);
            const float* uu = Us + (e * N + j) * 3;
            const float z0 = Z0c[j * 32 + lane];
            b0 = fmaf(v1 * uu[0], z0, b0);
            b1 = fmaf(v1 * uu[1], z0, b1);
            b2 = fmaf(v1 * uu[2], z0, b2);
            if (j == e) continue;
            const float* zs = Zsf + (j * 3) * 32 + lane;
            const float cr = uu[0] * (zr[3 * s][jj] - zs[0]) + uu[1] * (zr[3 * s + 1][jj] - zs[32]) +
                             uu[2] * (zr[3 * s + 2][jj] - zs[64]);
            const float w2 = SW1 ? W2[(jj * N + e) * 32 + lane] : w2v[SW1 ? 0 : jj];
            sv += (2.f * w2 + 4.f * v1 * Id[e * N + j]) * z0 + 2.f * v1 * cr;
          }
          SPb[(e * 3) * 32 + lane] = b0;
          SPb[(e * 3 + 1) * 32 + lane] = b1;
          SPb[(e * 3 + 2) * 32 + lane] = b2;
          SPc[e * 32 + lane] = sv;
        }
        __syncwarp();
        for (int i = 0; i < N; ++i) {
          float acc[CB];
#pragma unroll
          for (int q = 0; q < CB; ++q) acc[q] = 0.f;
          const float* wr = W0 + i * 32 + lane;
#pragma unroll
          for (int jj = 0; jj < NBS; ++jj) {
            const float w = wr[jj * N * 32];
#pragma unroll
            for (int q = 0; q < CB; ++q) acc[q] = fmaf(w, zr[q][jj], acc[q]);
          }
#pragma unroll
          for (int s = 0; s < EPT; ++s) {
            const int e = e0 + s;
            if (e >= N) break;
            // (a): -w'_ie z_e[0] u_ie,x (w'_ii = 0: nothing on the receiver's own channels)
            const float pa = (SW1 ? W1[(ja[s] * N + i) * 32 + lane] : w1_at(i, ja[s])) * za[s];
            const float* ue = Us + (i * N + e) * 3;
#pragma unroll
            for (int x = 0; x < 3; ++x) acc[3 * s + x] = fmaf(-pa, ue[x], acc[3 * s + x]);
            if (e == i) {  // (b): the receiver's own coordinates
#pragma unroll
              for (int x = 0; x < 3; ++x) acc[3 * s + x] += SPb[(i * 3 + x) * 32 + lane];
            }
          }
          const bool same = (i < n_up) == (pass == 0);
          const float nu = same ? nu_same : nu_opp;
          TO* o = mb + ((int64_t)i * C + c0) * 3 * D + (same ? 0 : D);
#pragma unroll
          for (int q = 0; q < CB; ++q)
            if (e0 + q / 3 < N) store_out(o + (int64_t)q * 3 * D, acc[q] * nu);
        }
      } else {
        // the value channel (z_j[0] from shared memory) and the Laplacian channel, with (c)
        float zv[NBS], zl[NBS];
#pragma unroll
        for (int jj = 0; jj < NBS; ++jj) {
          zv[jj] = jj < jn ? Z0c[(j0 + jj) * 32 + lane] : 0.f;
          zl[jj] = jj < jn ? Zb[((int64_t)(j0 + jj) * C + C - 1) * D] : 0.f;
        }
        for (int i = 0; i < N; ++i) {
          float av = 0.f, al = 0.f;
          const float* wr = W0 + i * 32 + lane;
#pragma unroll
          for (int jj = 0; jj < NBS; ++jj) {
            const float w = wr[jj * N * 32];
            av = fmaf(w, zv[jj], av);
            al = fmaf(w, zl[jj], al);
          }
          const bool same = (i < n_up) == (pass == 0);
          const float nu = same ? nu_same : nu_opp;
          store_out(mb + (int64_t)i * C * 3 * D + (same ? 0 : D), av * nu);
          LAP[i * 32 + lane] = al;  // completed with (c) after every task has written SPc
        }
      }
    }
    __syncthreads();
    // the Laplacian channel: contraction + (c)
    for (int i = warp; i < N; i += NW) {
      const bool same = (i < n_up) == (pass == 0);
      const float nu = same ? nu_same : nu_opp;
      const float al = LAP[i * 32 + lane] + SPc[i * 32 + lane];
      store_out(mb + ((int64_t)i * C + C - 1) * 3 * D + (same ? 0 : D), al * nu);
    }
    __syncthreads();  // the tables are rewritten by the next pass
  }
}

template <int NBS, int EPT, int NW, class TO>
cudaError_t launch_ml(const MLArgs& a, int64_t Bc, cudaStream_t s) {
  const MLSmem lay = ml_layout(a.N, NBS, a.stage_w1 != 0);
  auto kern = a.stage_w1 ? messages_large_kernel<NBS, EPT, NW, true, TO> : messages_large_kernel<NBS, EPT, NW, false, TO>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lay.total_bytes);
  if (e != cudaSuccess) return e;
  kern<<<dim3((unsigned)Bc, (unsigned)(a.D / kMLLanes)), NW * 32, lay.total_bytes, s>>>(a);
  return cudaGetLastError();
}

int ml_nbs(int nb) { return nb <= 8 ? 8 : nb <= 14 ? 14 : nb <= 16 ? 16 : 24; }

}  // namespace

bool messages_large_supported(const dq_handle_s& h, const FwdDims& d) {
  if (h.precision == DQ_FP64 || d.C != 3 * d.N + 2 || d.D % kMLLanes || d.N > kMLMaxN || d.N < 2) return false;
  const int nb = std::max(d.n_up, d.N - d.n_up);
  if (nb > 24) return false;
  const MLSmem l = ml_layout(d.N, ml_nbs(nb), false);
  return l.total_bytes <= 220 * 1024;
}

cudaError_t launch_messages_large(const dq_handle_s& h, const FwdDims& d, const float* params, int l,
                                  const float* Z, const float* ew, const float* geo, void* msg, bool bf16_out,
                                  cudaStream_t s) {
  if (d.Bc <= 0) return cudaSuccess;
  if (!messages_large_supported(h, d)) return cudaErrorInvalidValue;
  const int nb = std::max(d.n_up, d.N - d.n_up);
  const int nbs = ml_nbs(nb);
  MLArgs a{Z, ew, geo, params + h.off.layer[l].Y, h.d_pair_of, msg, d.N, d.n_up, d.M, d.C, d.D,
           h.edges.n_all, h.edges.n_ee, 1};
  if (ml_layout(d.N, nbs, true).total_bytes > 220 * 1024) a.stage_w1 = 0;
  // register tiles of sender slots x 3 EPT channels (72 to 84 values) in 16 warps of 128 registers
  if (nbs == 8)
    return bf16_out ? launch_ml<8, 3, 16, __nv_bfloat16>(a, d.Bc, s) : launch_ml<8, 3, 16, float>(a, d.Bc, s);
  if (nbs == 14)
    return bf16_out ? launch_ml<14, 2, 16, __nv_bfloat16>(a, d.Bc, s) : launch_ml<14, 2, 16, float>(a, d.Bc, s);
  if (nbs == 16)
    return bf16_out ? launch_ml<16, 1, 16, __nv_bfloat16>(a, d.Bc, s) : launch_ml<16, 1, 16, float>(a, d.Bc, s);
  return bf16_out ? launch_ml<24, 1, 16, __nv_bfloat16>(a, d.Bc, s) : launch_ml<24, 1, 16, float>(a, d.Bc, s);
}

}  // namespace dq
