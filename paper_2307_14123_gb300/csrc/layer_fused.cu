// One graph-convolution layer of the jets forward pass in one kernel (FP32
// and BF16 modes): the messages of Eq. 17 with their product-rule Jacobian and
// Laplacian channels, the update map W_g of Eq. 18 on the tensor cores, and
// the residual tanh update with its jet,
//   f <- f + tanh(u),  J(tanh u) = t' J(u),  L(tanh u) = t' L(u) + t'' sum_k J_k(u)^2,
//   u = W_g [m_par; m_anti; m_nuc] + b_g.
// The messages are the A operand of the MMAs and never leave the SM; the
// pre-activations u stay in tensor memory until the epilogue applies the
// update to f in place.  Per walker the kernel reads the node map z (written
// by the node-map GEMM), the filter jets, the geometry and f, and writes f.
//
// Rows of a tile: one walker, G = 128 / N consecutive node channels c and all
// N receivers i, row = (c - c0) N + i; a walker is ceil(C / G) tiles, which
// one CTA processes in channel order (the value channel first, the Laplacian
// last), so that the Laplacian cross terms and sum_k J_k(u)^2 accumulate on
// chip.  K steps: for each edge type t (same spin, opposite spin, nucleus)
// and 32-feature block, A[row][32] = m_i^t[c][32 features] as three TF32
// products with the W_g block (hi hi + hi lo + lo hi), or in BF16 mode as
// one product of BF16 operands (FP32 accumulation).
//
// Warp roles (16 warps, one CTA per SM, persistent over walkers):
//   warp 0      TMA: W_g hi/lo blocks (BF16: one block) and the z slab
//               z_j[c0 .. c0 + G)[32] of all senders into a 2-stage ring;
//   warp 1      MMA issue (tcgen05.mma kind::tf32, 128 x 128 x 8; BF16:
//               kind::f16, 128 x 128 x 16) into one of two tensor-memory
//               accumulators;
//   warps 2-3   idle;
//   warps 4-7   epilogue: tensor memory -> the pre-activations U in global memory;
//   warps 8-15  message producers: warp 8 + w owns two receivers of one spin
//               block (a half-warp each, two features per lane) and writes
//               their rows of the A block (TF32 high and low parts, 128-byte
//               swizzle; BF16: one part, 64-byte swizzle) from the z slab and
//               the filter jets, prefetching the next K step's filter lines
//               into L2.
// Every mbarrier wait is bounded (about one second); a timeout sets
// DQ_FLAG_TIMEOUT, the roles stop issuing work, and the tensor memory is
// released.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace dq {
namespace {
using namespace tcp;

constexpr int LF_BK = 32;                  // features per K step: one 128-byte row of the A block
constexpr int LF_D = 128;                  // embedding width (the MMA's N)
constexpr int LF_NFB = LF_D / LF_BK;       // feature blocks per edge type
constexpr int LF_KSTEPS = 2 * LF_NFB;      // K = 2 D: the electron-electron blocks of W_g
constexpr int LF_STAGES = 2;
constexpr int LF_UG = 2;                   // node channels per producer group
constexpr int LF_PROD = 16;                // producer warps at most (one per receiver)
// threads of the kernel for NB sender slots per spin block: 2 NB producer warps
// 16 warps in four warpgroups: TMA and MMA issue (and two idle warps), epilogue, and two
// warpgroups of producers (one warp per receiver pair).
constexpr int LF_THREADS = 512;
constexpr int LF_PROD_WARPS = 8;
constexpr int LF_MAX_N = 16;               // electrons (receivers per tile >= 8)
constexpr int LF_MAX_BLK = 8;              // electrons per spin block
constexpr int LF_MAX_M = 8;                // nuclei
constexpr uint32_t LF_TILE = 128 * LF_BK * 4;  // 16 KB: 128 rows x 32 FP32
constexpr uint32_t LF_STAGE = 4 * LF_TILE;     // A hi, A lo, B hi, B lo
constexpr int LF_ZBUF = 2;                     // z slabs in flight (one per feature block)
constexpr uint32_t LF_TMEM_ALLOC = 256;        // two 128-column accumulators

// Shared-memory layout (bytes from the 1024-aligned base).
constexpr uint32_t LF_OFF_Z = LF_STAGES * LF_STAGE;                                // [2][N][G][32] z slabs
constexpr uint32_t LF_OFF_ACCL = LF_OFF_Z + LF_ZBUF * LF_TILE;                      // [N][2][D] Laplacian cross terms
constexpr uint32_t LF_OFF_ST = LF_OFF_ACCL + LF_MAX_N * 2 * LF_D * 4;              // [4][32][33] transposes
constexpr uint32_t LF_OFF_GEO = LF_OFF_ST + 4 * 32 * 33 * 4;                       // per receiver tables
constexpr uint32_t LF_GEO_WARP = (LF_MAX_BLK * 2 + LF_MAX_M) * 8 * 4;              // rows x 8 floats
constexpr uint32_t LF_OFF_BAR = LF_OFF_GEO + LF_PROD * LF_GEO_WARP;
constexpr uint32_t LF_SMEM = 1024 + LF_OFF_BAR + 20 * 8 + 16;
static_assert(LF_SMEM <= 232448, "dynamic shared memory above the per-block limit");

struct LayerFusedArgs {
  const float* Z;       // [Bc][N][C][D] node map z_j (not read when z_const)
  const float* zv;      // [Bc][N][D] a copy of the value channel z_j[0] (U overwrites Z's)
  const float* z0;      // [2][D] node map of the two spin embeddings (z_const)
  const float* ew;      // [Bc][E][3][D] filter jets: w, dw/dd, d2w/dd2
  const float* geo;     // [Bc][E][4] distance and unit vector of every edge
  const int* pair_of;   // [N][N] edge of (i, j), -1 on the diagonal
  float* U;             // [Bc][N][C][D] W_g's electron-electron blocks times the messages (may be Z:
                        // a tile's rows are written after the last read of its z slab)
  int64_t Bc;
  int N, n_up, M, C, E, n_ee, G, n_tiles;
  int z_const;
  int n_prod;  // producer warps (receiver pairs), at most LF_PROD_WARPS
};

__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

// x rounded to the nearest TF32 value (11 significant bits) by Veltkamp splitting: three FP32
// operations, ties to even; the low part of a TF32 pair is rounded the same way, so that the
// tensor cores (which read the top 19 bits of an operand) see it in full.
__device__ __forceinline__ float tf32_split_hi(float x) {
  const float t = __fmul_rn(x, 8193.f);
  return __fsub_rn(t, __fsub_rn(t, x));
}

// One lane's two messages (features 2 fp and 2 fp + 1 of its K step) into row `row` of the A
// block.  FP32 mode: TF32 high and low parts, each rounded to 11 significant bits, in two
// 128-row x 128-byte tiles (128-byte swizzle: 16-byte chunk c of row r at c ^ (r & 7)).  BF16
// mode: one BF16 pair (round to nearest even) in a 128-row x 64-byte tile (64-byte swizzle:
// chunk c of row r at c ^ ((r >> 1) & 3)).
template <bool BF>
__device__ __forceinline__ void store_a(uint8_t* a_hi, uint8_t* a_lo, int row, int fp, float2 m) {
  if constexpr (BF) {
    const uint32_t o = (uint32_t)row * 64u + ((((uint32_t)fp >> 2) ^ (((uint32_t)row >> 1) & 3u)) << 4) +
                       ((uint32_t)(fp & 3) << 2);
    *reinterpret_cast<__nv_bfloat162*>(a_hi + o) = __floats2bfloat162_rn(m.x, m.y);
  } else {
    float2 hi, lo;
    hi.x = tf32_split_hi(m.x);
    hi.y = tf32_split_hi(m.y);
    lo.x = tf32_split_hi(__fsub_rn(m.x, hi.x));
    lo.y = tf32_split_hi(__fsub_rn(m.y, hi.y));
    const uint32_t o = (uint32_t)row * 128u + ((((uint32_t)fp >> 1) ^ (uint32_t)(row & 7)) << 4) +
                       ((uint32_t)(fp & 1) << 3);
    *reinterpret_cast<float2*>(a_hi + o) = hi;
    *reinterpret_cast<float2*>(a_lo + o) = lo;
  }
}

// NB: sender slots per spin block (at least the larger block's electron count); ZC: constant
// node channels (layer 0 with spin embeddings); BF: BF16 operands (one MMA product per K
// step) instead of the 3 x TF32 products.
template <int NB, bool ZC, bool BF>
__global__ void __launch_bounds__(LF_THREADS, 1)
    layer_fused_kernel(const __grid_constant__ LayerFusedArgs a, const __grid_constant__ CUtensorMap map_whi,
                       const __grid_constant__ CUtensorMap map_wlo, const __grid_constant__ CUtensorMap map_z,
                       const __grid_constant__ CUtensorMap map_wbf, unsigned int* __restrict__ status) {
  extern __shared__ __align__(1024) uint8_t lf_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(lf_smem_raw) + 1023) & ~(uintptr_t)1023);
  float* accL = reinterpret_cast<float*>(smem + LF_OFF_ACCL);
  float* stg = reinterpret_cast<float*>(smem + LF_OFF_ST);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + LF_OFF_BAR);
  uint64_t* conv = full + LF_STAGES;
  uint64_t* empty = conv + LF_STAGES;
  uint64_t* acc_full = empty + LF_STAGES;  // [2]
  uint64_t* acc_empty = acc_full + 2;      // [2]
  uint64_t* zfull = acc_empty + 2;         // [LF_ZBUF]
  uint64_t* zempty = zfull + LF_ZBUF;      // [LF_ZBUF]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(zempty + LF_ZBUF);
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int N = a.N, C = a.C, G = a.G, n_tiles = a.n_tiles;
  const uint32_t zbytes = (uint32_t)(LF_BK * G * N * 4);
  const int n_prod = a.n_prod;  // producer warps: one per receiver pair

  if (threadIdx.x == 0) {
    for (int s = 0; s < LF_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], n_prod);  // one arrival per producer warp
      mbar_init(&empty[s], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&acc_full[q], 1);
      mbar_init(&acc_empty[q], 4);  // one arrival per epilogue warp
    }
    for (int q = 0; q < LF_ZBUF; ++q) {
      mbar_init(&zfull[q], 1);
      mbar_init(&zempty[q], n_prod);  // released by every producer warp after its last use
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  // z slabs and cross-term sums start as zeros: slab rows past a box (never written by TMA) are
  // read, with weight zero, by the sender slots past a spin block
  for (uint32_t e = threadIdx.x; e < (LF_OFF_ST - LF_OFF_Z) / 4; e += blockDim.x)
    reinterpret_cast<float*>(smem + LF_OFF_Z)[e] = 0.f;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(LF_TMEM_ALLOC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int64_t g_ks = 0, zi = 0;
      for (int64_t b = blockIdx.x; b < a.Bc && !s_abort; b += gridDim.x) {
        for (int g = 0; g < n_tiles && !s_abort; ++g) {
          for (int ks = 0; ks < LF_KSTEPS && !s_abort; ++ks, ++g_ks) {
            const int fb = ks / 2, t = ks % 2;
            if (t == 0 && !a.z_const) {  // the feature block's z slab, used by its first two K steps
              const int zb = (int)(zi % LF_ZBUF);
              const int64_t u = zi / LF_ZBUF;
              if (u >= 1 && !wait_or_abort(&zempty[zb], (uint32_t)((u - 1) & 1), &s_abort)) {
                s_abort = 1;
                break;
              }
              mbar_expect_tx(&zfull[zb], zbytes);
              tma_load_3d(smem + LF_OFF_Z + zb * LF_TILE, &map_z, fb * LF_BK, (int)(b * N), g * G, &zfull[zb]);
              ++zi;
            }
            const int s = (int)(g_ks % LF_STAGES);
            const int64_t u = g_ks / LF_STAGES;
            if (u >= 1 && !wait_or_abort(&empty[s], (uint32_t)((u - 1) & 1), &s_abort)) {
              s_abort = 1;
              break;
            }
            uint8_t* st = smem + s * LF_STAGE;
            if (BF) {  // the BF16 block of W_g: 128 rows x 64 bytes
              mbar_expect_tx(&full[s], LF_TILE / 2);
              tma_load_2d(st + 2 * LF_TILE, &map_wbf, t * LF_D + fb * LF_BK, 0, &full[s]);
            } else {
              mbar_expect_tx(&full[s], 2 * LF_TILE);
              tma_load_2d(st + 2 * LF_TILE, &map_whi, t * LF_D + fb * LF_BK, 0, &full[s]);
              tma_load_2d(st + 3 * LF_TILE, &map_wlo, t * LF_D + fb * LF_BK, 0, &full[s]);
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      constexpr uint32_t idesc = BF ? tc_idesc(128, LF_D) : t3_idesc(128, LF_D);
      int64_t g_ks = 0, lt = 0;
      bool ok = true;
      for (int64_t b = blockIdx.x; b < a.Bc && ok && !s_abort; b += gridDim.x) {
        for (int g = 0; g < n_tiles && ok; ++g, ++lt) {
          const int q = (int)(lt & 1);
          const int64_t v = lt >> 1;
          if (v >= 1 && !wait_or_abort(&acc_empty[q], (uint32_t)((v - 1) & 1), &s_abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(q * LF_D);
          for (int ks = 0; ks < LF_KSTEPS; ++ks, ++g_ks) {
            const int s = (int)(g_ks % LF_STAGES);
            if (!wait_or_abort(&conv[s], (uint32_t)((g_ks / LF_STAGES) & 1), &s_abort)) {
              ok = false;
              break;
            }
            tc_fence_after();
            uint8_t* st = smem + s * LF_STAGE;
            const uint32_t ah = smem_u32(st), al = smem_u32(st + LF_TILE);
            const uint32_t bh = smem_u32(st + 2 * LF_TILE), bl = smem_u32(st + 3 * LF_TILE);
            if constexpr (BF) {  // two K = 16 products per 32-feature step
#pragma unroll
              for (int kk = 0; kk < LF_BK / 16; ++kk)
                umma_bf16(d, sw64_desc(ah + kk * 32), sw64_desc(bh + kk * 32), idesc, (ks | kk) ? 1u : 0u);
            } else {
#pragma unroll
              for (int kk = 0; kk < LF_BK / 8; ++kk) {
                const uint32_t o = kk * 32;
                umma_tf32(d, sw128_desc(ah + o), sw128_desc(bh + o), idesc, (ks | kk) ? 1u : 0u);
                umma_tf32(d, sw128_desc(ah + o), sw128_desc(bl + o), idesc, 1u);
                umma_tf32(d, sw128_desc(al + o), sw128_desc(bh + o), idesc, 1u);
              }
            }
            umma_commit(&empty[s]);
          }
          if (!ok) break;
          umma_commit(&acc_full[q]);
        }
      }
      if (!ok) s_abort = 1;
    }
  } else if (warp >= 8) {
    if (warp - 8 >= n_prod) goto done;  // no receiver pair for this warp
    // ---- message producers: warp 8 + w owns receiver pair w (two receivers of one spin block);
    // lane (h, fp) = (lane / 16, lane % 16) computes features f0 + 2 fp and f0 + 2 fp + 1 of
    // receiver i_h.  The last pair of an odd block repeats its receiver in the second half,
    // which computes but never writes. ----
    const int w = warp - 8;
    const int h = lane >> 4, fp = lane & 15;
    const int n_up = a.n_up, M = a.M, E = a.E, n_ee = a.n_ee;
    const int pairs_up = (n_up + 1) >> 1;
    int i = w < pairs_up ? 2 * w + h : n_up + 2 * (w - pairs_up) + h;
    const bool writer = w < pairs_up ? i < n_up : i < N;
    if (!writer) i -= 1;
    const bool up = i < n_up;
    // geometry of receiver i, once per walker: per sender slot k of the same spin block (k < 8),
    // of the other block (8 <= k < 16) and per nucleus (16 <= k): the edge index (as float bits),
    // the unit vector u_ij and 1 / d_ij
    float* gt = reinterpret_cast<float*>(smem + LF_OFF_GEO + i * LF_GEO_WARP);
    constexpr int kRows = LF_MAX_BLK * 2 + LF_MAX_M;
    int64_t g_ks = 0, zi = 0;
    bool ok = true;
    // the filter-jet lines of K step (t, f0) into L2: lane fp < 8 sender slot fp's value,
    // 8 <= fp its first derivative
    auto prefetch_filters = [&](const float* ew_b, int t, int f0) {
      const int k = fp & 7, jet = fp >> 3;
      const int row = (t == 0 ? 0 : LF_MAX_BLK) + k;
      const int edge = __float_as_int(gt[row * 8]);
      if (edge >= 0)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(ew_b + ((int64_t)edge * 3 + jet) * LF_D + f0));
    };
    for (int64_t b = blockIdx.x; b < a.Bc && ok; b += gridDim.x) {
      const float* geo_b = a.geo + b * E * 4;
      const float* ew_b = a.ew + b * (int64_t)E * 3 * LF_D;
      const float* zv_b = a.zv + b * (int64_t)N * LF_D;
      if (writer) {
        for (int k = fp; k < kRows; k += 16) {
          float* row = gt + k * 8;
          int edge = -1;
          float sg = 1.f;
          if (k < 2 * LF_MAX_BLK) {
            const bool same = k < LF_MAX_BLK;
            const int j0 = (up == same) ? 0 : n_up, j1 = (up == same) ? n_up : N;
            const int j = j0 + (k % LF_MAX_BLK);
            if (j < j1 && j != i) {
              edge = a.pair_of[i * N + j];
              sg = i < j ? 1.f : -1.f;
            }
          } else if (k - 2 * LF_MAX_BLK < M) {
            edge = n_ee + i * M + (k - 2 * LF_MAX_BLK);
          }
          if (edge >= 0) {
            const float* gg = geo_b + (int64_t)edge * 4;
            row[0] = __int_as_float(edge);
            row[1] = sg * gg[1];
            row[2] = sg * gg[2];
            row[3] = sg * gg[3];
            row[4] = 1.f / gg[0];
          } else {
            row[0] = __int_as_float(-1);
            row[1] = row[2] = row[3] = row[4] = 0.f;
          }
        }
      }
      __syncwarp();
      prefetch_filters(ew_b, 0, 0);
      for (int g = 0; g < n_tiles && ok; ++g) {
        const int c0 = g * G;
        const int c1 = min(C, c0 + G);
        for (int ks = 0; ks < LF_KSTEPS; ++ks, ++g_ks) {
          const int s = (int)(g_ks % LF_STAGES);
          const int fb = ks / 2, t = ks % 2;
          const int f0 = fb * LF_BK;
          const int fl = f0 + 2 * fp;  // this lane's first feature
          // electron-electron messages of type t: senders j = j0 + k, k < NB
          const bool same = t == 0;
          const int j0 = (up == same) ? 0 : n_up, j1 = (up == same) ? n_up : N;
          const float* gs = gt + (same ? 0 : LF_MAX_BLK) * 8;
          // the step's filter jets and, past tile 0, the senders' z_j[0] (global loads issued
          // before the waits, so that their latency overlaps them); slots without an edge read
          // edge 0 and are masked below
          float2 wv[NB], w1[NB], z0v[NB];
#pragma unroll
          for (int k = 0; k < NB; ++k) {
            const int edge = __float_as_int(gs[k * 8]);
            const float* wp = ew_b + (int64_t)(edge >= 0 ? edge : 0) * 3 * LF_D + fl;
            wv[k] = __ldg(reinterpret_cast<const float2*>(wp));
            w1[k] = __ldg(reinterpret_cast<const float2*>(wp + LF_D));
            const int j = min(j0 + k, N - 1);
            if (ZC)
              z0v[k] = __ldg(reinterpret_cast<const float2*>(a.z0 + (j < n_up ? 0 : LF_D) + fl));
            else if (c0 > 0)
              z0v[k] = __ldg(reinterpret_cast<const float2*>(zv_b + (int64_t)j * LF_D + fl));
          }
          // the Laplacian channel's w'' lines into L2 ahead of their use at the end of the step
          if (c1 == C && fp < NB) {
            const int edge = __float_as_int(gs[fp * 8]);
            if (edge >= 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(ew_b + ((int64_t)edge * 3 + 2) * LF_D + f0));
          }
          if (!wait_or_abort(&full[s], (uint32_t)((g_ks / LF_STAGES) & 1), &s_abort)) {
            ok = false;
            break;
          }
          uint8_t* a_hi = smem + s * LF_STAGE;
          uint8_t* a_lo = a_hi + LF_TILE;
          const int zb = (int)(zi % LF_ZBUF);
          const float* zs = reinterpret_cast<const float*>(smem + LF_OFF_Z + zb * LF_TILE);  // [c - c0][j][32]
          if (!ZC && !wait_or_abort(&zfull[zb], (uint32_t)((zi / LF_ZBUF) & 1), &s_abort)) {
            ok = false;
            break;
          }
          const int n_send = same ? (j1 - j0) - 1 : (j1 - j0);
          const float nu = 1.f / (float)(n_send > 1 ? n_send : 1);
          // the next K step's filter lines into L2 while this one is produced
          if (ks + 1 < LF_KSTEPS) prefetch_filters(ew_b, (ks + 1) % 2, ((ks + 1) / 2) * LF_BK);
          else if (g + 1 < n_tiles) prefetch_filters(ew_b, 0, 0);
#pragma unroll
          for (int k = 0; k < NB; ++k) {
            const bool v = __float_as_int(gs[k * 8]) >= 0;
            const int j = min(j0 + k, N - 1);
            if (!ZC && c0 == 0) z0v[k] = *reinterpret_cast<const float2*>(zs + j * LF_BK + 2 * fp);
            wv[k] = v ? wv[k] : make_float2(0.f, 0.f);
            w1[k] = v ? w1[k] : make_float2(0.f, 0.f);
            z0v[k] = v ? z0v[k] : make_float2(0.f, 0.f);
          }
          float* acl = accL + (i * 2 + t) * LF_D + fl;
          float2 accv = g == 0 ? make_float2(0.f, 0.f) : *reinterpret_cast<const float2*>(acl);
          {
            // the receiver's own coordinates, for both halves at once (no divergence on i):
            // m_i[c] = sum_j w_ij z_j[c] + sum_j w'_ij u_ij,x z_j[0], c = 1 + 3 i + x, and the Laplacian
            // cross term 2 sum_j w'_ij u_ij,x dz_j/dr_i,x (before the channel loop, whose Laplacian
            // channel reads the cross terms)
            const int cb = 1 + 3 * i;
            const bool any_own = cb + 2 >= c0 && cb < c1;
            if (__any_sync(0xffffffffu, any_own)) {
#pragma unroll
              for (int x = 0; x < 3; ++x) {
                const int c = cb + x;
                const bool act = c >= c0 && c < c1;
                const float* zr = zs + ((act ? c - c0 : 0) * N + j0) * LF_BK + 2 * fp;
                float2 m = make_float2(0.f, 0.f), cr = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                  const float ux = gs[k * 8 + 1 + x];
                  const float2 ak = make_float2(w1[k].x * ux, w1[k].y * ux);
                  m.x = fmaf(ak.x, z0v[k].x, m.x);
                  m.y = fmaf(ak.y, z0v[k].y, m.y);
                  if (!ZC) {
                    const float2 z = *reinterpret_cast<const float2*>(zr + k * LF_BK);
                    m.x = fmaf(wv[k].x, z.x, m.x);
                    m.y = fmaf(wv[k].y, z.y, m.y);
                    cr.x = fmaf(ak.x, z.x, cr.x);
                    cr.y = fmaf(ak.y, z.y, cr.y);
                  }
                }
                if (act) {
                  accv.x = fmaf(2.f, cr.x, accv.x);
                  accv.y = fmaf(2.f, cr.y, accv.y);
                  if (writer) {
                    m.x *= nu;
                    m.y *= nu;
                    store_a<BF>(a_hi, a_lo, (c - c0) * N + i, fp, m);
                  }
                }
              }
            }
          }
          const float* zrow = zs + j0 * LF_BK + 2 * fp;  // channel c0's senders
          int row = i;                                    // A row of (c0, i)
          int e = c0 >= 1 ? (c0 - 1) / 3 : -1, x = c0 >= 1 ? (c0 - 1) - 3 * e : 2;  // electron, axis of c0
          int ke_c = -1;                                  // the sender slot whose w' and z_j[0] are cached
          float2 w1e = make_float2(0.f, 0.f), z0e = make_float2(0.f, 0.f);
          // channels in groups of LF_UG: the loads and multiply-add chains of a group overlap
          for (int cg = c0; cg < c1; cg += LF_UG, zrow += LF_UG * N * LF_BK) {
            float2 zc[LF_UG][NB], mm[LF_UG];
#pragma unroll
            for (int u = 0; u < LF_UG; ++u) {
              // rows past c1 stay inside the z buffers (finite data) and their sums are dropped
#pragma unroll
              for (int k = 0; k < NB; ++k)
                zc[u][k] = ZC ? make_float2(0.f, 0.f) : *reinterpret_cast<const float2*>(zrow + (u * N + k) * LF_BK);
            }
#pragma unroll
            for (int u = 0; u < LF_UG; ++u) {
              float2 m0 = make_float2(0.f, 0.f), m1 = make_float2(0.f, 0.f);
              if (!ZC || (cg + u == 0)) {
#pragma unroll
                for (int k = 0; k < NB; k += 2) {
                  const float2 z = ZC ? z0v[k] : zc[u][k];
                  m0.x = fmaf(wv[k].x, z.x, m0.x);
                  m0.y = fmaf(wv[k].y, z.y, m0.y);
                  if (k + 1 < NB) {
                    const float2 z1 = ZC ? z0v[k + 1] : zc[u][k + 1];
                    m1.x = fmaf(wv[k + 1].x, z1.x, m1.x);
                    m1.y = fmaf(wv[k + 1].y, z1.y, m1.y);
                  }
                }
              }
              mm[u] = make_float2(m0.x + m1.x, m0.y + m1.y);
            }
#pragma unroll
            for (int u = 0; u < LF_UG; ++u) {
              const int c = cg + u;
              if (c >= c1) break;
              float2 m = mm[u];
              if (c >= 1 && c < C - 1) {
                if (e >= j0 && e < j1) {
                  // a sender's coordinate: -w'_ie u_ie,x z_e[0]; Laplacian cross term
                  // -2 w'_ie u_ie,x dz_e/dr_e,x (zero for the receiver's own slot, whose weights
                  // are masked); the slot's registers are picked once per electron
                  const int ke = e - j0;
                  if (ke != ke_c) {
                    ke_c = ke;
                    w1e = w1[0];
                    z0e = z0v[0];
#pragma unroll
                    for (int k = 1; k < NB; ++k)
                      if (ke == k) {
                        w1e = w1[k];
                        z0e = z0v[k];
                      }
                  }
                  const float ux = gs[ke * 8 + 1 + x];
                  const float2 ak = make_float2(w1e.x * ux, w1e.y * ux);
                  m.x = fmaf(-ak.x, z0e.x, m.x);
                  m.y = fmaf(-ak.y, z0e.y, m.y);
                  if (!ZC) {
                    const float2 zce = *reinterpret_cast<const float2*>(zrow + (u * N + ke) * LF_BK);
                    accv.x = fmaf(-2.f * ak.x, zce.x, accv.x);
                    accv.y = fmaf(-2.f * ak.y, zce.y, accv.y);
                  }
                }
              } else if (c == C - 1) {
                // sum_j (2 w''_ij + 4 w'_ij / d_ij) z_j[0] + the accumulated cross terms
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                  const int edge = __float_as_int(gs[k * 8]);
                  const float2 w2 = edge >= 0
                                        ? __ldg(reinterpret_cast<const float2*>(ew_b + ((int64_t)edge * 3 + 2) * LF_D + fl))
                                        : make_float2(0.f, 0.f);
                  const float id = 4.f * gs[k * 8 + 4];
                  m.x = fmaf(fmaf(2.f, w2.x, id * w1[k].x), z0v[k].x, m.x);
                  m.y = fmaf(fmaf(2.f, w2.y, id * w1[k].y), z0v[k].y, m.y);
                }
                m.x += accv.x;
                m.y += accv.y;
              }
              m.x *= nu;
              m.y *= nu;
              if (writer && e != i)  // (the receiver's own channels were formed above)
                store_a<BF>(a_hi, a_lo, row, fp, m);
              row += N;
              if (++x == 3) {
                x = 0;
                ++e;
              }
            }
          }
          if (writer) *reinterpret_cast<float2*>(acl) = accv;
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // A block visible to the tensor cores
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&conv[s])) : "memory");
          if (t == 1 && !ZC) {  // the z slab's last use: release it to the TMA thread
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&zempty[zb])) : "memory");
            ++zi;
          }
        }
      }
    }
    if (!ok) s_abort = 1;
  } else if (warp >= 4) {
    // ---- epilogue warps 4..7: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 ----
    // Per 32-feature chunk: the warp's 32 rows of the accumulator through a shared-memory
    // transpose, stored as full 128-byte lines of U (the electron-nucleus part, un, is added by
    // the kernel that follows).
    const int q = warp % 4;
    float(*stw)[33] = reinterpret_cast<float(*)[33]>(stg + q * 32 * 33);
    int64_t lt = 0;
    for (int64_t b = blockIdx.x; b < a.Bc; b += gridDim.x) {
      float* Ub = a.U + b * (int64_t)N * C * LF_D;
      for (int g = 0; g < n_tiles; ++g, ++lt) {
        const int acc_i = (int)(lt & 1);
        const int c0 = g * G;
        const int c1 = min(C, c0 + G);
        const int nrows = (c1 - c0) * N;
        bool live = wait_or_abort(&acc_full[acc_i], (uint32_t)((lt >> 1) & 1), &s_abort) && !s_abort;
        live = __all_sync(0xffffffffu, live);  // warp-uniform: the tensor-memory loads are warp-wide
        if (!live) s_abort = 1;
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(acc_i * LF_D) + ((uint32_t)(q * 32) << 16);
        const int cc_first = (q * 32) / N, i_first = (q * 32) - cc_first * N;
        for (int d0 = 0; d0 < LF_D && live; d0 += 32) {
          uint32_t v[32];
          tmem_ld32(acc + (uint32_t)d0, v);
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) stw[lane][jj] = __uint_as_float(v[jj]);
          __syncwarp();
          int cc = cc_first, ii = i_first;
          for (int rr = 0; rr < 32; ++rr) {
            if (q * 32 + rr >= nrows) break;
            Ub[((int64_t)ii * C + c0 + cc) * LF_D + d0 + lane] = stw[rr][lane];
            if (++ii == N) {
              ii = 0;
              ++cc;
            }
          }
          __syncwarp();
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[acc_i])) : "memory");
      }
    }
  }
done:
  __syncthreads();
  if (s_abort && threadIdx.x == 0) atomicOr(status, (unsigned)DQ_FLAG_TIMEOUT);
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(LF_TMEM_ALLOC) : "memory");
}

// Electron-nucleus messages of Eq. 17 on the channels where they are non-zero (d_iI depends on
// r_i alone): mn[b][i][5][D] = (value, the three coordinates of r_i, Laplacian) of
// (1/M) sum_I w(d_iI) Y_I with the jets of w; one block per (walker, receiver), a thread per feature.
__global__ void nucleus_messages_kernel(const float* __restrict__ ew, const float* __restrict__ geo,
                                        const float* __restrict__ Y, int N, int M, int E, int n_ee,
                                        float* __restrict__ mn) {
  const int64_t bi = blockIdx.x;
  const int64_t b = bi / N;
  const int i = (int)(bi % N), d = threadIdx.x;
  float nv = 0.f, nx = 0.f, ny = 0.f, nz = 0.f, nl = 0.f;
  for (int I = 0; I < M; ++I) {
    const int64_t e = b * E + n_ee + (int64_t)i * M + I;
    const float* g = geo + e * 4;
    const float* w = ew + e * 3 * LF_D + d;
    const float y = __ldg(Y + I * LF_D + d);
    const float w0 = __ldg(w), w1 = __ldg(w + LF_D), w2 = __ldg(w + 2 * LF_D);
    nv += w0 * y;
    nx += w1 * g[1] * y;
    ny += w1 * g[2] * y;
    nz += w1 * g[3] * y;
    nl += (w2 + 2.f * w1 / g[0]) * y;
  }
  const float nu = 1.f / (float)M;
  float* o = mn + bi * 5 * LF_D + d;
  o[0] = nv * nu;
  o[LF_D] = nx * nu;
  o[2 * LF_D] = ny * nu;
  o[3 * LF_D] = nz * nu;
  o[4 * LF_D] = nl * nu;
}

// zv[b][j][:] = Z[b][j][0][:]: the value channel of the node map, which the producers read
// while the epilogue overwrites Z with the pre-activations.
__global__ void value_channel_kernel(const float* __restrict__ Z, int64_t BN, int C, float* __restrict__ zv) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= BN * LF_D) return;
  zv[e] = Z[(e / LF_D) * C * LF_D + (e % LF_D)];
}

// U[b][i][c][:] += un[b][i][slot][:] on the channels where the electron-nucleus messages are
// non-zero: slot 0 the value channel (b_g included), 1..3 the receiver's own coordinates, 4 the
// Laplacian.  One block per (walker, receiver), a thread per feature.
__global__ void add_nucleus_part_kernel(const float* __restrict__ un, int N, int C, float* __restrict__ U) {
  const int64_t bi = blockIdx.x;
  const int i = (int)(bi % N), d = threadIdx.x;
  const float* src = un + bi * 5 * LF_D + d;
  float* dst = U + bi * C * LF_D + d;
  const int ch[5] = {0, 1 + 3 * i, 2 + 3 * i, 3 + 3 * i, C - 1};
#pragma unroll
  for (int k = 0; k < 5; ++k) dst[(int64_t)ch[k] * LF_D] += src[(int64_t)k * LF_D];
}

// The BF16 copy of W_g [D][3 D] as dims {3 D, D}, box {32, 128}: 64-byte rows, 64-byte swizzle.
bool map_w_bf(CUtensorMap* m, const void* W, int D) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(3 * D), (cuuint64_t)D};
  const cuuint64_t strides[1] = {(cuuint64_t)(3 * D) * 2};
  const cuuint32_t box[2] = {LF_BK, 128};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(W), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool map_w(CUtensorMap* m, const float* W, int D) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(3 * D), (cuuint64_t)D};
  const cuuint64_t strides[1] = {(cuuint64_t)(3 * D) * 4};
  const cuuint32_t box[2] = {LF_BK, 128};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(W), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// z [Bc][N][C][D] as dims {D, N Bc, C} (sender before channel); box {32 features, N senders,
// G channels}, so that the slab in shared memory is [channel][sender][32]; channels past C read zeros.
bool map_z(CUtensorMap* m, const float* Z, int64_t Bc, int N, int C, int D, int G) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)D, (cuuint64_t)(N * Bc), (cuuint64_t)C};
  const cuuint64_t strides[2] = {(cuuint64_t)C * D * 4, (cuuint64_t)D * 4};
  const cuuint32_t box[3] = {LF_BK, (cuuint32_t)N, (cuuint32_t)G};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(Z), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

using KernT = void (*)(LayerFusedArgs, CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, unsigned int*);

template <bool BF>
KernT pick_kernel(int nb, bool z_const) {
  if (z_const)
    return nb <= 2 ? layer_fused_kernel<2, true, BF> : nb <= 4 ? layer_fused_kernel<4, true, BF>
           : nb <= 5 ? layer_fused_kernel<5, true, BF> : nb <= 7 ? layer_fused_kernel<7, true, BF>
                     : layer_fused_kernel<8, true, BF>;
  return nb <= 2 ? layer_fused_kernel<2, false, BF> : nb <= 4 ? layer_fused_kernel<4, false, BF>
         : nb <= 5 ? layer_fused_kernel<5, false, BF> : nb <= 7 ? layer_fused_kernel<7, false, BF>
                   : layer_fused_kernel<8, false, BF>;
}

}  // namespace

bool layer_fused_supported(const dq_handle_s& h) {
  return (h.precision == DQ_FP32 || h.precision == DQ_BF16_MIXED) && h.D == LF_D && h.N >= 1 && h.N <= LF_MAX_N && h.n_up <= LF_MAX_BLK &&
         h.n_dn <= LF_MAX_BLK && h.M >= 1 && h.M <= LF_MAX_M;
}

cudaError_t launch_layer_fused(const dq_handle_s& h, const FwdDims& d, const float* params, int l, bool z_const,
                               float* Z, const float* z0, const float* ew, const float* geo, float* mn,
                               const float* wg_hi, const float* wg_lo, const void* wg_bf, cudaStream_t s) {
  if (d.Bc <= 0) return cudaSuccess;
  if (!layer_fused_supported(h) || d.C != 3 * d.N + 2) return cudaErrorInvalidValue;
  const auto& y = h.off.layer[l];
  const int64_t rows5 = d.Bc * d.N * 5;
  float* un = mn + rows5 * LF_D;
  float* zv = un + rows5 * LF_D;
  if (!z_const) {
    value_channel_kernel<<<(unsigned)((d.Bc * d.N * LF_D + 255) / 256), 256, 0, s>>>(Z, d.Bc * d.N, d.C, zv);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
  }
  // electron-nucleus part of the update map: u_n = W_g[:, 2D:3D] m_n (+ b_g on the value slot)
  nucleus_messages_kernel<<<(unsigned)(d.Bc * d.N), LF_D, 0, s>>>(ew, geo, params + y.Y, d.N, d.M, h.edges.n_all,
                                                                  h.edges.n_ee, mn);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  T3JobDesc jn{mn, rows5, 1, 0, LF_D, LF_D, wg_hi + 2 * LF_D, wg_lo + 2 * LF_D, LF_D, params + y.b_g, 5, un, LF_D,
               0, false, 3 * LF_D};
  e = gemm_tf32x3_tc_jobs(&jn, 1, h.d_status, s);
  if (e != cudaSuccess) return e;
  LayerFusedArgs a{};
  a.Z = Z;
  a.zv = zv;
  a.z0 = z0;
  a.ew = ew;
  a.geo = geo;
  a.pair_of = h.d_pair_of;
  a.U = Z;
  a.Bc = d.Bc;
  a.N = d.N;
  a.n_up = d.n_up;
  a.M = d.M;
  a.C = d.C;
  a.E = h.edges.n_all;
  a.n_ee = h.edges.n_ee;
  a.G = std::min(128 / d.N, d.C);
  a.n_tiles = (d.C + a.G - 1) / a.G;
  a.z_const = z_const ? 1 : 0;
  CUtensorMap mhi, mlo, mz, mbf;
  if (!map_w(&mhi, wg_hi, LF_D) || !map_w(&mlo, wg_lo, LF_D)) return cudaErrorInvalidValue;
  // BF16 operands when the BF16 copy of W_g is given (otherwise mbf is a copy of the FP32 map, unread)
  if (wg_bf ? !map_w_bf(&mbf, wg_bf, LF_D) : !map_w(&mbf, wg_hi, LF_D)) return cudaErrorInvalidValue;
  // with constant node channels the z slabs are never loaded; their maps are built on W (any valid map)
  if (!(z_const ? map_w(&mz, wg_hi, LF_D) : map_z(&mz, Z, d.Bc, d.N, d.C, LF_D, a.G))) return cudaErrorInvalidValue;
  const int nb = std::max(h.n_up, h.n_dn);
  const KernT kern = wg_bf ? pick_kernel<true>(nb, z_const) : pick_kernel<false>(nb, z_const);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LF_SMEM);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = d.Bc < sms ? d.Bc : sms;
  a.n_prod = (h.n_up + 1) / 2 + (h.n_dn + 1) / 2;  // receiver pairs of the two spin blocks
  if (a.n_prod > LF_PROD_WARPS) return cudaErrorInvalidValue;
  kern<<<(unsigned)grid, LF_THREADS, LF_SMEM, s>>>(a, mhi, mlo, mz, mbf, h.d_status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  add_nucleus_part_kernel<<<(unsigned)(d.Bc * d.N), LF_D, 0, s>>>(un, d.N, d.C, Z);
  return cudaGetLastError();
}

}  // namespace dq
