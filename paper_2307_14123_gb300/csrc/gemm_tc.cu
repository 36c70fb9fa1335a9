// BF16 tensor-core GEMM for the embedding layers (5th-generation tensor cores).
//
//   Y[r][n] = sum_k X[r][k] W[n][k] + (r % bias_period == 0 ? bias[n] : 0)
//
// X [rows][K] and W [n_out][K] are BF16, K-major (row stride ldx, K); Y is
// FP32 with row stride ldy.  This is the linear map of the graph-convolution
// update (W_g, Eq. 18) and of the node map (W_h, Eq. 17) acting on all
// value / Jacobian / Laplacian channels at once: the rows are the channels of
// every node of every walker, so one launch is one large dense contraction.
//
// A persistent grid (one CTA per SM) walks the 128 x 128 output tiles:
//   * warp 0, lane 0 streams 128 x 64 tiles of X and W into a 3-stage ring of
//     shared-memory buffers with TMA (cp.async.bulk.tensor, 128-byte swizzle),
//     completing on "full" mbarriers;
//   * warp 1, lane 0 issues tcgen05.mma (kind::f16, BF16 inputs, FP32
//     accumulator in tensor memory, M = 128, N = 128, K = 16 per instruction)
//     and releases each stage with tcgen05.commit on its "empty" mbarrier;
//   * warps 2..5 read a finished accumulator back with tcgen05.ld (a warp
//     reaches the 32 tensor-memory lanes of its index modulo 4) and store FP32
//     while the next tile accumulates in the second accumulator.
// Rows beyond `rows` and columns beyond n_out are zero-filled by TMA and not
// stored.  Every mbarrier wait is bounded (about one second of clock); on
// timeout the kernel sets DQ_FLAG_TIMEOUT in the status word, skips the rest
// and still releases its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace dq {
namespace {
using namespace tcp;

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_STAGES = 3;
constexpr uint32_t TC_TILE_A = TC_BM * TC_BK * 2;  // 16 KB
constexpr uint32_t TC_TILE_B = TC_BN * TC_BK * 2;  // 16 KB
constexpr uint32_t TC_TMEM_COLS = 128;
// Persistent kernel: CTA c processes output tiles c, c + gridDim.x, ... in
// order (tile = m-tile * n_tiles + n-tile).  Warp roles: warp 0 lane 0 TMA
// producer (continuous stream of k-blocks across tiles); warp 1 lane 0 MMA
// issuer; warps 2..5 epilogue.  Two accumulators in tensor memory (2 x 128
// columns): the MMA warp fills one while the epilogue warps drain the other
// (acc_full / acc_empty mbarriers), so the epilogue of a tile overlaps the
// loads and MMAs of the next.
// Epilogue store of a 32 x 32 FP32 block that a warp holds one row per lane
// (after tmem_ld32: lane t has row t, columns 0..31), through a padded
// shared-memory transpose so that every store instruction writes 32
// consecutive columns of one row (one full 128-byte line).  my_row: this
// lane's destination row pointer at the block's first column (nullptr: row
// outside the output); my_bias: that row takes the bias; bn: the bias of this
// lane's column; col_ok: this lane's column is inside the output.
__device__ __forceinline__ void store_block_32x32(const uint32_t (&v)[32], float (*st)[33], int lane, float* my_row,
                                                  bool my_bias, float bn, bool col_ok, bool accumulate = false) {
#pragma unroll
  for (int j = 0; j < 32; ++j) st[lane][j] = __uint_as_float(v[j]);
  __syncwarp();
  const unsigned long long pr = reinterpret_cast<unsigned long long>(my_row);
  const uint32_t plo = (uint32_t)pr, phi = (uint32_t)(pr >> 32), fb = my_bias ? 1u : 0u;
#pragma unroll 4
  for (int rr = 0; rr < 32; ++rr) {
    const uint32_t lo = __shfl_sync(0xffffffffu, plo, rr), hi = __shfl_sync(0xffffffffu, phi, rr);
    const uint32_t b = __shfl_sync(0xffffffffu, fb, rr);
    float* y = reinterpret_cast<float*>(((unsigned long long)hi << 32) | lo);
    const float val = st[rr][lane] + (b ? bn : 0.f);
    if (y != nullptr && col_ok) y[lane] = accumulate ? y[lane] + val : val;
  }
  __syncwarp();
}

constexpr int TC_THREADS = 192;
constexpr uint32_t TC_TMEM_ALLOC = 2 * TC_TMEM_COLS;

__global__ void __launch_bounds__(TC_THREADS, 1)
    gemm_bf16_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        int64_t rows, int n_out, int K, const float* __restrict__ bias, int bias_period,
                        float* __restrict__ Y, int64_t ldy, unsigned int* __restrict__ status) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + TC_STAGES * TC_TILE_A;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + TC_STAGES * TC_TILE_B);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* acc_full = empty + TC_STAGES;  // [2]
  uint64_t* acc_empty = acc_full + 2;      // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  __shared__ volatile int s_abort;
  __shared__ float ep_stage[4][32][33];  // epilogue transpose, one block per epilogue warp

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nk = K / TC_BK;
  const int n_tiles_n = (n_out + TC_BN - 1) / TC_BN;
  const int64_t n_tiles = ((rows + TC_BM - 1) / TC_BM) * n_tiles_n;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_ALLOC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int64_t g = 0;   // k-blocks issued so far
      for (int64_t t = blockIdx.x; t < n_tiles && !s_abort; t += gridDim.x) {
        const int64_t m0 = (t / n_tiles_n) * TC_BM;
        const int n0 = (int)(t % n_tiles_n) * TC_BN;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = (int)(g % TC_STAGES);
          const int64_t u = g / TC_STAGES;
          if (u >= 1 && !mbar_wait(&empty[s], (uint32_t)((u - 1) & 1))) {
            s_abort = 1;
            break;
          }
          mbar_expect_tx(&full[s], TC_TILE_A + TC_TILE_B);
          tma_load_2d(sA + s * TC_TILE_A, &tmA, kb * TC_BK, (int)m0, &full[s]);
          tma_load_2d(sB + s * TC_TILE_B, &tmB, kb * TC_BK, n0, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      constexpr uint32_t idesc = tc_idesc(TC_BM, TC_BN);
      int64_t g = 0, lt = 0;
      for (int64_t t = blockIdx.x; t < n_tiles && !s_abort; t += gridDim.x, ++lt) {
        const int a = (int)(lt & 1);
        const int64_t v = lt >> 1;
        if (v >= 1 && !mbar_wait(&acc_empty[a], (uint32_t)((v - 1) & 1))) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(a * TC_TMEM_COLS);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = (int)(g % TC_STAGES);
          if (!mbar_wait(&full[s], (uint32_t)((g / TC_STAGES) & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + s * TC_TILE_A), b0 = smem_u32(sB + s * TC_TILE_B);
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk)
            umma_bf16(d, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc, (kb | kk) ? 1u : 0u);
          umma_commit(&empty[s]);
        }
        if (!ok) {
          s_abort = 1;
          break;
        }
        umma_commit(&acc_full[a]);
      }
    }
  } else {
    // Epilogue warps 2..5: warp w reads tensor-memory lanes 32 (w % 4) .. + 31.
    const int q = warp % 4;
    float(*st)[33] = ep_stage[warp - 2];
    int64_t lt = 0;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++lt) {
      const int a = (int)(lt & 1);
      const int64_t v = lt >> 1;
      if (!mbar_wait(&acc_full[a], (uint32_t)(v & 1))) {
        s_abort = 1;
        break;
      }
      tc_fence_after();
      const int64_t m0 = (t / n_tiles_n) * TC_BM;
      const int n0 = (int)(t % n_tiles_n) * TC_BN;
      const int64_t row = m0 + q * 32 + lane;
      const bool add_bias = bias != nullptr && (row % bias_period) == 0;
      float* yrow = row < rows ? Y + row * ldy + n0 : nullptr;
      for (int c0 = 0; c0 < TC_BN; c0 += 32) {
        uint32_t vv[32];
        tmem_ld32(tmem + (uint32_t)(a * TC_TMEM_COLS) + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, vv);
        const int n = n0 + c0 + lane;
        const bool col_ok = n < n_out;
        store_block_32x32(vv, st, lane, yrow ? yrow + c0 : nullptr, add_bias, bias != nullptr && col_ok ? bias[n] : 0.f,
                          col_ok);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[a])) : "memory");
    }
  }
  __syncthreads();
  if (s_abort && threadIdx.x == 0) atomicOr(status, (unsigned)DQ_FLAG_TIMEOUT);
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_ALLOC) : "memory");
}

// ---------------------------------------------------------------------------
// FP32-accurate variant for the FP32 mode: 3 x TF32 splitting.
//   x = x_big + x_small with x_big = tf32(x), x_small = tf32(x - x_big);
//   x . w ~= x_big w_big + x_big w_small + x_small w_big   (error ~ 2^-22 |x||w|)
// W is split once per call (split_tf32_kernel).  The FP32 X tile arrives by
// TMA; four converter warps split it in shared memory (x_big in place, x_small
// into a second buffer at the same positions: the split is elementwise, so the
// 128-byte-swizzled layout carries over) and release it to the MMA warp after a
// proxy fence.  Three tcgen05.mma.kind::tf32 (K = 8 per instruction) per
// 8-element slice accumulate into one FP32 accumulator in tensor memory.
// Warps: 0 TMA, 1 MMA, 2..5 and 10..13 epilogue (column halves), 6..9 converter.
// ---------------------------------------------------------------------------
constexpr int T3_BK = 32;                            // FP32 elements per 128-byte row
constexpr int T3_STAGES = 2;
constexpr int T3_SUB = 2;                               // 128-row blocks per tile (share the W tile)
constexpr uint32_t T3_TMEM_ALLOC = 2 * T3_SUB * 128;    // double-buffered, T3_SUB accumulators each
constexpr uint32_t T3_TILE_A = TC_BM * T3_BK * 4;    // 16 KB
constexpr uint32_t T3_TILE_B = TC_BN * T3_BK * 4;    // 16 KB
constexpr int T3_THREADS = 320;     // the row-reduction kernel: TMA, MMA, 4 epilogue, 4 converter warps
constexpr int T3J_THREADS = 448;    // the job-list GEMM: 4 more epilogue warps (10..13)

__global__ void split_tf32_kernel(const float* __restrict__ W, float* __restrict__ big, float* __restrict__ small,
                                  int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float x = W[e], b = tf32_rn(x);
  big[e] = b;
  small[e] = tf32_rn(x - b);
}

// Split of the transpose: W [rows][cols] -> big, small [cols][rows] (the B
// operand of X W, whose reduction index is W's row index).
__global__ void split_tf32_t_kernel(const float* __restrict__ W, int rows, int cols, float* __restrict__ big,
                                    float* __restrict__ small) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    tile[k][threadIdx.x] = r < rows && c < cols ? W[(int64_t)r * cols + c] : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (c < cols && r < rows) {
      const float x = tile[threadIdx.x][k], b = tf32_rn(x);
      big[(int64_t)c * rows + r] = b;
      small[(int64_t)c * rows + r] = tf32_rn(x - b);
    }
  }
}

// One launch runs a list of GEMMs (jobs): the edge filters of every edge type,
// the orbitals of both spins, or one step of several molecules.  Tiles of all
// jobs form one sequence that the persistent CTAs take in turn; a job's tiles
// are contiguous, so every role finds the job of a tile by its prefix counts.
// A 128-row block holds rb rows of each of sb = TC_BM / rb segments (rb <
// TC_BM only if seg_rows <= rb), or a TC_BM-row block of one segment.  A tile is
// T3_SUB such blocks sharing the W tile; each has its own accumulator.
// Reads of the parameter block at run-time offsets are slow (measured: a job
// table read that way cost a third of the GEMM's speed at K = 128), so the
// roles that run per K block or per output element read it at compile-time
// offsets only: the producer's TMA loads and the epilogue are templates on the
// job index, reached through a switch.  The job lookup itself reads a copy of
// the scalar fields that each CTA keeps in shared memory.
struct T3Fields {
  const float* bias;
  float* Y;
  int64_t seg_rows, n_seg, ldy, y_seg_stride;
  int64_t rb_per_seg, n_mblk, tile_end;  // tile_end: tiles of jobs 0 .. this one
  int rb, sb, n_out, nk, n_tiles_n, bias_period, accumulate;
};
struct T3Job {
  CUtensorMap a, bb, bs;  // X (segmented rows), W big, W small
  T3Fields f;
};
constexpr int kT3MaxJobs = 16;
struct T3Jobs {
  T3Job j[kT3MaxJobs];
  int n;
};
__device__ __forceinline__ int t3_job(const T3Fields* sj, int n, int64_t t, int64_t& tl) {
  int m = 0;
  while (m + 1 < n && t >= sj[m].tile_end) ++m;
  tl = t - (m > 0 ? sj[m - 1].tile_end : 0);
  return m;
}
// TMA loads of one K block of job M's tile (A blocks of T3_SUB segments, W big and small).
template <int M>
__device__ __forceinline__ void t3_issue(const T3Jobs& jobs, uint8_t* a_dst, uint8_t* bb_dst, uint8_t* bs_dst,
                                         int x, const int* m0, const int* seg, int n0, uint64_t* bar) {
  asm volatile("// job %0" ::"n"(M));  // keeps the 16 cases of the switch apart
#pragma unroll
  for (int h = 0; h < T3_SUB; ++h) tma_load_3d(a_dst + h * T3_TILE_A, &jobs.j[M].a, x, m0[h], seg[h], bar);
  tma_load_2d(bb_dst, &jobs.j[M].bb, x, n0, bar);
  tma_load_2d(bs_dst, &jobs.j[M].bs, x, n0, bar);
}

// Epilogue of one tile of job M (the job's fields read at compile-time offsets
// of the parameter block): TMEM -> registers -> shared-memory transpose -> Y.
template <int M>
__device__ __forceinline__ void t3_epi_tile(const T3Jobs& jobs, int64_t tl, uint32_t acc, int q, int lane,
                                            float (*st)[17], int c_lo, int c_hi, uint64_t* rows_tab) {
  asm volatile("// job %0" ::"n"(M));  // keeps the 16 cases of the switch apart
  const T3Fields& J = jobs.j[M].f;
  const int n_tiles_n = J.n_tiles_n, rb = J.rb, sbk = J.sb, bias_period = J.bias_period, n_out = J.n_out;
  const int accumulate = J.accumulate;
  const int64_t rb_per_seg = J.rb_per_seg, n_mblk = J.n_mblk, seg_rows = J.seg_rows, n_seg = J.n_seg;
  const int64_t ldy = J.ldy, y_seg_stride = J.y_seg_stride;
  float* const Y = J.Y;
  const float* const bias = J.bias;
  const int64_t mp = tl / n_tiles_n;
  const int n0 = (int)(tl % n_tiles_n) * TC_BN;
  const int tr = q * 32 + lane;  // row of the 128-row block
  const int half = lane >> 4, col = lane & 15;  // store phase: two rows of 16 columns per instruction
#pragma unroll 1
  for (int h = 0; h < T3_SUB; ++h) {
    const int64_t mb = mp * T3_SUB + h;
    const int64_t seg = (mb / rb_per_seg) * sbk + tr / rb;
    const int64_t row = (mb % rb_per_seg) * rb + tr % rb;  // row within the segment
    const bool add_bias = bias != nullptr && (row % bias_period) == 0;
    float* yrow = mb < n_mblk && row < seg_rows && seg < n_seg ? Y + seg * y_seg_stride + row * ldy + n0 : nullptr;
    // the warp's 32 row pointers (bit 0: add the bias), read back as shared-memory broadcasts
    __syncwarp();
    rows_tab[lane] = reinterpret_cast<uint64_t>(yrow) | (add_bias ? 1ull : 0ull);
    __syncwarp();
    for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
      uint32_t vv[16];
      tmem_ld16(acc + (uint32_t)(h * TC_TMEM_COLS) + (uint32_t)c0, vv);
#pragma unroll
      for (int j = 0; j < 16; ++j) st[lane][j] = __uint_as_float(vv[j]);
      __syncwarp();
      const int n = n0 + c0 + col;
      const bool col_ok = n < n_out;
      const float bn = bias != nullptr && col_ok ? bias[n] : 0.f;
#pragma unroll 8
      for (int rr = 0; rr < 32; rr += 2) {
        const uint64_t e = rows_tab[rr + half];
        float* y = reinterpret_cast<float*>(e & ~1ull);
        const float val = st[rr + half][col] + ((e & 1ull) ? bn : 0.f);
        if (y != nullptr && col_ok) y[c0 + col] = accumulate ? y[c0 + col] + val : val;
      }
      __syncwarp();
    }
  }
}

__global__ void __launch_bounds__(T3J_THREADS, 1)
    gemm_tf32x3_tc_kernel(const __grid_constant__ T3Jobs jobs, unsigned int* __restrict__ status) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  // per stage: [x half 0, x half 1] (x_big after conversion), [x_small half 0, half 1], w_big, w_small
  uint8_t* sA = smem;
  uint8_t* sAs = sA + T3_STAGES * T3_SUB * T3_TILE_A;
  uint8_t* sBb = sAs + T3_STAGES * T3_SUB * T3_TILE_A;
  uint8_t* sBs = sBb + T3_STAGES * T3_TILE_B;
  uint64_t* full = reinterpret_cast<uint64_t*>(sBs + T3_STAGES * T3_TILE_B);
  uint64_t* conv = full + T3_STAGES;
  uint64_t* empty = conv + T3_STAGES;
  uint64_t* acc_full = empty + T3_STAGES;  // [2]
  uint64_t* acc_empty = acc_full + 2;      // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  __shared__ volatile int s_abort;
  __shared__ float ep_stage[8][32][17];  // epilogue transposes, one block per epilogue warp
  __shared__ uint64_t ep_rows[8][32];     // epilogue row pointers

  __shared__ T3Fields sj[kT3MaxJobs];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n_jobs = jobs.n;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < kT3MaxJobs; ++k)
      if (k < n_jobs) sj[k] = jobs.j[k].f;
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < T3_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 4);  // one arrival per converter warp
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 8);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(T3_TMEM_ALLOC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t n_tiles = sj[n_jobs - 1].tile_end;  // (job, row-block pair, column block)

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int64_t g = 0;
      for (int64_t t = blockIdx.x; t < n_tiles && !s_abort; t += gridDim.x) {
        int64_t tl;
        const int jm = t3_job(sj, n_jobs, t, tl);
        const T3Fields& J = sj[jm];
        const int n_tiles_n = J.n_tiles_n, nk = J.nk, rb = J.rb, sbk = J.sb;
        const int64_t rb_per_seg = J.rb_per_seg;
        const int64_t mp = tl / n_tiles_n;
        const int n0 = (int)(tl % n_tiles_n) * TC_BN;
        int seg[T3_SUB], m0[T3_SUB];
#pragma unroll
        for (int h = 0; h < T3_SUB; ++h) {  // first segment and row of each 128-row block (past the end: zero fill)
          const int64_t mb = mp * T3_SUB + h;
          seg[h] = (int)(mb / rb_per_seg) * sbk;
          m0[h] = (int)(mb % rb_per_seg) * rb;
        }
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = (int)(g % T3_STAGES);
          const int64_t u = g / T3_STAGES;
          if (u >= 1 && !mbar_wait(&empty[s], (uint32_t)((u - 1) & 1))) {
            s_abort = 1;
            break;
          }
          mbar_expect_tx(&full[s], T3_SUB * T3_TILE_A + 2 * T3_TILE_B);
          uint8_t* const ad = sA + s * T3_SUB * T3_TILE_A;
          uint8_t* const bbd = sBb + s * T3_TILE_B;
          uint8_t* const bsd = sBs + s * T3_TILE_B;
          const int x = kb * T3_BK;
          switch (jm) {
#define T3_CASE(M) \
  case M: t3_issue<M>(jobs, ad, bbd, bsd, x, m0, seg, n0, &full[s]); break;
            T3_CASE(0) T3_CASE(1) T3_CASE(2) T3_CASE(3) T3_CASE(4) T3_CASE(5) T3_CASE(6) T3_CASE(7)
            T3_CASE(8) T3_CASE(9) T3_CASE(10) T3_CASE(11) T3_CASE(12) T3_CASE(13) T3_CASE(14) T3_CASE(15)
#undef T3_CASE
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      constexpr uint32_t idesc = t3_idesc(TC_BM, TC_BN);
      int64_t g = 0, lt = 0;
      for (int64_t t = blockIdx.x; t < n_tiles && !s_abort; t += gridDim.x, ++lt) {
        const int a = (int)(lt & 1);
        const int64_t v = lt >> 1;
        if (v >= 1 && !mbar_wait(&acc_empty[a], (uint32_t)((v - 1) & 1))) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        int64_t tl;
        const int nk = sj[t3_job(sj, n_jobs, t, tl)].nk;
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = (int)(g % T3_STAGES);
          if (!mbar_wait(&conv[s], (uint32_t)((g / T3_STAGES) & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t bb = smem_u32(sBb + s * T3_TILE_B), bs = smem_u32(sBs + s * T3_TILE_B);
#pragma unroll
          for (int h = 0; h < T3_SUB; ++h) {
            const uint32_t d = tmem + (uint32_t)((a * T3_SUB + h) * TC_TMEM_COLS);
            const uint32_t ab = smem_u32(sA + (s * T3_SUB + h) * T3_TILE_A);
            const uint32_t as_ = smem_u32(sAs + (s * T3_SUB + h) * T3_TILE_A);
#pragma unroll
            for (int kk = 0; kk < T3_BK / 8; ++kk) {
              const uint32_t o = kk * 32;
              umma_tf32(d, sw128_desc(ab + o), sw128_desc(bb + o), idesc, (kb | kk) ? 1u : 0u);
              umma_tf32(d, sw128_desc(ab + o), sw128_desc(bs + o), idesc, 1u);
              umma_tf32(d, sw128_desc(as_ + o), sw128_desc(bb + o), idesc, 1u);
            }
          }
          umma_commit(&empty[s]);
        }
        if (!ok) {
          s_abort = 1;
          break;
        }
        umma_commit(&acc_full[a]);
      }
    }
  } else if (warp >= 6 && warp < 10) {
    // Converter warps 6..9: split each FP32 X tile into TF32 big (in place) and small.
    const int ct = threadIdx.x - 6 * 32;  // 0..127
    int64_t g = 0;
    for (int64_t t = blockIdx.x; t < n_tiles && !s_abort; t += gridDim.x) {
      int64_t tl;
      const int nk = sj[t3_job(sj, n_jobs, t, tl)].nk;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = (int)(g % T3_STAGES);
        if (!mbar_wait(&full[s], (uint32_t)((g / T3_STAGES) & 1))) {
          s_abort = 1;
          break;
        }
        float4* src = reinterpret_cast<float4*>(sA + s * T3_SUB * T3_TILE_A);
        float4* dst = reinterpret_cast<float4*>(sAs + s * T3_SUB * T3_TILE_A);
#pragma unroll 4
        for (int j = 0; j < (int)(T3_SUB * T3_TILE_A / 16 / 128); ++j) {
          const int idx = j * 128 + ct;
          const float4 x = src[idx];
          float4 b, sm;
          b.x = tf32_rn(x.x);
          b.y = tf32_rn(x.y);
          b.z = tf32_rn(x.z);
          b.w = tf32_rn(x.w);
          sm.x = tf32_rn(x.x - b.x);
          sm.y = tf32_rn(x.y - b.y);
          sm.z = tf32_rn(x.z - b.z);
          sm.w = tf32_rn(x.w - b.w);
          src[idx] = b;
          dst[idx] = sm;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&conv[s])) : "memory");
      }
    }
  } else {
    // Epilogue warps 2..5 and 10..13: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 of each
    // accumulator, columns 0..63 (warps 2..5) or 64..127 (warps 10..13).
    const int q = warp % 4;
    const int eg = warp >= 10 ? 1 : 0, ei = eg * 4 + (warp - (eg ? 10 : 2));
    float(*st)[17] = ep_stage[ei];
    int64_t lt = 0;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++lt) {
      const int a = (int)(lt & 1);
      const int64_t v = lt >> 1;
      if (!mbar_wait(&acc_full[a], (uint32_t)(v & 1))) {
        s_abort = 1;
        break;
      }
      tc_fence_after();
      int64_t tl;
      const int jm = t3_job(sj, n_jobs, t, tl);
      const uint32_t acc = tmem + (uint32_t)(a * T3_SUB * TC_TMEM_COLS) + ((uint32_t)(q * 32) << 16);
      switch (jm) {
#define T3_EPI(M) \
  case M: t3_epi_tile<M>(jobs, tl, acc, q, lane, st, 64 * eg, 64 * eg + 64, ep_rows[ei]); break;
        T3_EPI(0) T3_EPI(1) T3_EPI(2) T3_EPI(3) T3_EPI(4) T3_EPI(5) T3_EPI(6) T3_EPI(7)
        T3_EPI(8) T3_EPI(9) T3_EPI(10) T3_EPI(11) T3_EPI(12) T3_EPI(13) T3_EPI(14) T3_EPI(15)
#undef T3_EPI
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[a])) : "memory");
    }
  }
  __syncthreads();
  if (s_abort && threadIdx.x == 0) atomicOr(status, (unsigned)DQ_FLAG_TIMEOUT);
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T3_TMEM_ALLOC) : "memory");
}

// ---------------------------------------------------------------------------
// Row reductions on the tensor cores (weight gradients of the reverse pass):
//   part[split][o][a] = sum over the split's rows r of X[r][o] * Y[r][a]
// as 3 x TF32 products with the reduction (row) index as the MMA's K.  Rows
// come in segments (one per walker); a K step takes 32 rows: rb rows of each
// of 32 / rb segments.  X and Y tiles arrive by TMA as [32 rows][128 columns]
// (rows are the slow index of both operands); the converter warps transpose
// them into the K-major 128-byte-swizzled layout of the MMA operands while
// splitting into TF32 high and low parts.  Work items are (o tile, a tile,
// split); each writes its partial tile, and reduce_splits adds the splits in
// a fixed order.  With colpart, the converter threads also sum the X columns
// they transpose (FP32, rows in order) and the a-tile-0 items write
// colpart[split][o] = sum over the split's rows of X[r][o]: the bias-type
// gradient of the same adjoint, without a second pass over X.
// Warps: 0 TMA, 1 MMA, 2..5 epilogue, 6..9 converter.
// ---------------------------------------------------------------------------
constexpr int TN_BK = 32;                                  // rows per K step
constexpr uint32_t TN_TILE = TC_BM * TN_BK * 4;            // 16 KB: one 128 x 32 FP32 tile
constexpr int TN_TSTAGES = 2, TN_OSTAGES = 2;

__global__ void __launch_bounds__(T3_THREADS, 1)
    gemm_tn_tf32x3_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
                          int64_t rps, int64_t n_seg, int rb, int n_o, int n_a, int64_t splits, int64_t kps,
                          float* __restrict__ part, float* __restrict__ colpart, unsigned int* __restrict__ status) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sT = smem;                                   // [tstage][X tile, Y tile] as loaded: [32 rows][128]
  uint8_t* sO = sT + TN_TSTAGES * 2 * TN_TILE;          // [ostage][A hi, A lo, B hi, B lo] K-major, swizzled
  uint64_t* full = reinterpret_cast<uint64_t*>(sO + TN_OSTAGES * 4 * TN_TILE);
  uint64_t* tfree = full + TN_TSTAGES;
  uint64_t* ready = tfree + TN_TSTAGES;
  uint64_t* ofree = ready + TN_OSTAGES;
  uint64_t* acc_full = ofree + TN_OSTAGES;  // [2]
  uint64_t* acc_empty = acc_full + 2;       // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  __shared__ volatile int s_abort;
  __shared__ float ep_stage[4][32][33];

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int sb = TN_BK / rb;
  const int64_t rbps = (rps + rb - 1) / rb;                 // row blocks per segment
  const int64_t ktot = ((n_seg + sb - 1) / sb) * rbps;      // K steps in all
  const int tiles_m = (n_o + TC_BM - 1) / TC_BM, tiles_n = (n_a + TC_BN - 1) / TC_BN;
  const int64_t n_items = (int64_t)tiles_m * tiles_n * splits;
  auto item_range = [&](int64_t it, int& m0, int& n0, int64_t& sp, int64_t& k0, int64_t& k1) {
    sp = it % splits;
    const int64_t mn = it / splits;
    m0 = (int)(mn / tiles_n) * TC_BM;
    n0 = (int)(mn % tiles_n) * TC_BN;
    k0 = sp * kps;
    k1 = k0 + kps < ktot ? k0 + kps : ktot;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < TN_TSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&tfree[s], 4);
    }
    for (int s = 0; s < TN_OSTAGES; ++s) {
      mbar_init(&ready[s], 4);
      mbar_init(&ofree[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_ALLOC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int64_t g = 0;
      for (int64_t it = blockIdx.x; it < n_items && !s_abort; it += gridDim.x) {
        int m0, n0;
        int64_t sp, k0, k1;
        item_range(it, m0, n0, sp, k0, k1);
        for (int64_t ks = k0; ks < k1; ++ks, ++g) {
          const int s = (int)(g % TN_TSTAGES);
          const int64_t u = g / TN_TSTAGES;
          if (u >= 1 && !mbar_wait(&tfree[s], (uint32_t)((u - 1) & 1))) {
            s_abort = 1;
            break;
          }
          const int seg = (int)((ks / rbps) * sb), r0 = (int)((ks % rbps) * rb);
          mbar_expect_tx(&full[s], 2 * TN_TILE);
          tma_load_3d(sT + (s * 2 + 0) * TN_TILE, &tmX, m0, r0, seg, &full[s]);
          tma_load_3d(sT + (s * 2 + 1) * TN_TILE, &tmY, n0, r0, seg, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      constexpr uint32_t idesc = t3_idesc(TC_BM, TC_BN);
      int64_t g = 0, lt = 0;
      for (int64_t it = blockIdx.x; it < n_items && !s_abort; it += gridDim.x, ++lt) {
        int m0, n0;
        int64_t sp, k0, k1;
        item_range(it, m0, n0, sp, k0, k1);
        const int a = (int)(lt & 1);
        const int64_t v = lt >> 1;
        if (v >= 1 && !mbar_wait(&acc_empty[a], (uint32_t)((v - 1) & 1))) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(a * TC_TMEM_COLS);
        bool ok = true;
        for (int64_t ks = k0; ks < k1; ++ks, ++g) {
          const int s = (int)(g % TN_OSTAGES);
          if (!mbar_wait(&ready[s], (uint32_t)((g / TN_OSTAGES) & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ah = smem_u32(sO + (s * 4 + 0) * TN_TILE), al = smem_u32(sO + (s * 4 + 1) * TN_TILE);
          const uint32_t bh = smem_u32(sO + (s * 4 + 2) * TN_TILE), bl = smem_u32(sO + (s * 4 + 3) * TN_TILE);
#pragma unroll
          for (int kk = 0; kk < TN_BK / 8; ++kk) {
            const uint32_t o = kk * 32;
            umma_tf32(d, sw128_desc(ah + o), sw128_desc(bh + o), idesc, (ks > k0 || kk) ? 1u : 0u);
            umma_tf32(d, sw128_desc(ah + o), sw128_desc(bl + o), idesc, 1u);
            umma_tf32(d, sw128_desc(al + o), sw128_desc(bh + o), idesc, 1u);
          }
          umma_commit(&ofree[s]);
        }
        if (!ok) {
          s_abort = 1;
          break;
        }
        umma_commit(&acc_full[a]);
      }
    }
  } else if (warp >= 6) {
    // Converter warps: warp w transposes columns 32 w .. 32 w + 31 of both tiles.
    const int w = warp - 6;
    const int col = 32 * w + lane;
    int64_t g = 0;
    for (int64_t it = blockIdx.x; it < n_items && !s_abort; it += gridDim.x) {
      int m0, n0;
      int64_t sp, k0, k1;
      item_range(it, m0, n0, sp, k0, k1);
      float csum = 0.f;  // sum of this thread's X column over the item's rows
      for (int64_t ks = k0; ks < k1; ++ks, ++g) {
        const int ts = (int)(g % TN_TSTAGES), os = (int)(g % TN_OSTAGES);
        if (!mbar_wait(&full[ts], (uint32_t)((g / TN_TSTAGES) & 1)) ||
            (g >= TN_OSTAGES && !mbar_wait(&ofree[os], (uint32_t)((g / TN_OSTAGES - 1) & 1)))) {
          s_abort = 1;
          break;
        }
#pragma unroll
        for (int op = 0; op < 2; ++op) {  // X -> A, Y -> B
          const float* src = reinterpret_cast<const float*>(sT + (ts * 2 + op) * TN_TILE);
          uint8_t* hi = sO + (os * 4 + 2 * op) * TN_TILE;
          uint8_t* lo = hi + TN_TILE;
#pragma unroll
          for (int rq = 0; rq < TN_BK / 4; ++rq) {
            float4 h, l;
            float x;
            x = src[(4 * rq + 0) * TC_BM + col]; h.x = tf32_rn(x); l.x = tf32_rn(x - h.x);
            if (op == 0) csum += x;
            x = src[(4 * rq + 1) * TC_BM + col]; h.y = tf32_rn(x); l.y = tf32_rn(x - h.y);
            if (op == 0) csum += x;
            x = src[(4 * rq + 2) * TC_BM + col]; h.z = tf32_rn(x); l.z = tf32_rn(x - h.z);
            if (op == 0) csum += x;
            x = src[(4 * rq + 3) * TC_BM + col]; h.w = tf32_rn(x); l.w = tf32_rn(x - h.w);
            if (op == 0) csum += x;
            // K-major, 128-byte swizzle: row col, 16-byte chunk rq at chunk rq ^ (col % 8)
            const uint32_t off = (uint32_t)col * 128u + ((uint32_t)(rq ^ (col & 7)) << 4);
            *reinterpret_cast<float4*>(hi + off) = h;
            *reinterpret_cast<float4*>(lo + off) = l;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ready[os])) : "memory");
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tfree[ts])) : "memory");
        }
      }
      if (colpart != nullptr && n0 == 0 && m0 + col < n_o && !s_abort) colpart[sp * n_o + m0 + col] = csum;
    }
  } else {
    // Epilogue warps 2..5: rows o, columns a of the partial tile
    const int q = warp % 4;
    float(*st)[33] = ep_stage[warp - 2];
    int64_t lt = 0;
    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x, ++lt) {
      int m0, n0;
      int64_t sp, k0, k1;
      item_range(it, m0, n0, sp, k0, k1);
      const int a = (int)(lt & 1);
      const int64_t v = lt >> 1;
      if (!mbar_wait(&acc_full[a], (uint32_t)(v & 1))) {
        s_abort = 1;
        break;
      }
      tc_fence_after();
      const int o = m0 + q * 32 + lane;
      float* yrow = o < n_o ? part + (sp * n_o + o) * (int64_t)n_a + n0 : nullptr;
      for (int c0 = 0; c0 < TC_BN; c0 += 32) {
        uint32_t vv[32];
        tmem_ld32(tmem + (uint32_t)(a * TC_TMEM_COLS) + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, vv);
        store_block_32x32(vv, st, lane, yrow ? yrow + c0 : nullptr, false, 0.f, n0 + c0 + lane < n_a);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[a])) : "memory");
    }
  }
  __syncthreads();
  if (s_abort && threadIdx.x == 0) atomicOr(status, (unsigned)DQ_FLAG_TIMEOUT);
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_ALLOC) : "memory");
}

bool make_map(CUtensorMap* m, const void* base, int64_t rows, int K, int64_t ld, int box_rows, bool fp32 = false) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const int el = fp32 ? 4 : 2;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * el};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / el), (cuuint32_t)box_rows};  // one 128-byte row per box row
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
// FP32 rows in segments: dims {K, seg_rows, n_seg}, box {32, 128, 1}
bool make_map_seg_f32(CUtensorMap* m, const void* base, int64_t seg_rows, int64_t n_seg, int K, int64_t ld,
                      int64_t seg_stride, int rb) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)seg_rows, (cuuint64_t)n_seg};
  const cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)seg_stride * 4};
  const cuuint32_t box[3] = {32, (cuuint32_t)rb, (cuuint32_t)(TC_BM / rb)};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
constexpr size_t t3_smem_bytes() {
  return 1024 + T3_STAGES * (2 * T3_SUB * T3_TILE_A + 2 * T3_TILE_B) + (3 * T3_STAGES + 4) * 8 + 16;
}

constexpr size_t tc_smem_bytes() { return 1024 + TC_STAGES * (TC_TILE_A + TC_TILE_B) + (2 * TC_STAGES + 4) * 8 + 16; }

}  // namespace

cudaError_t gemm_bf16_tc(const void* X, int64_t rows, int K, int64_t ldx, const void* W, int n_out, const float* bias,
                         int bias_period, float* Y, int64_t ldy, unsigned int* status, cudaStream_t s) {
  if (rows <= 0 || n_out <= 0) return cudaSuccess;
  if (K % TC_BK || ldx % 8 || (uintptr_t)X % 16 || (uintptr_t)W % 16 || bias_period <= 0)
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, X, rows, K, ldx, TC_BM) || !make_map(&mb, W, n_out, K, K, TC_BN)) return cudaErrorInvalidValue;
  const size_t smem = tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = ((rows + TC_BM - 1) / TC_BM) * ((n_out + TC_BN - 1) / TC_BN);
  const int64_t grid = tiles < sms ? tiles : sms;
  gemm_bf16_tc_kernel<<<(unsigned)grid, TC_THREADS, smem, s>>>(ma, mb, rows, n_out, K, bias, bias_period, Y, ldy,
                                                             status);
  return cudaGetLastError();
}

cudaError_t split_tf32(const float* W, float* big, float* small, int64_t n, cudaStream_t s) {
  split_tf32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(W, big, small, n);
  return cudaGetLastError();
}

cudaError_t split_tf32_t(const float* W, int rows, int cols, float* big, float* small, cudaStream_t s) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  split_tf32_t_kernel<<<grid, dim3(32, 8), 0, s>>>(W, rows, cols, big, small);
  return cudaGetLastError();
}

cudaError_t gemm_tf32x3_tc_jobs(const T3JobDesc* d, int n, unsigned int* status, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = t3_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(gemm_tf32x3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  T3Jobs J;
  J.n = 0;
  int64_t tiles = 0;
  auto flush = [&]() -> cudaError_t {
    if (J.n == 0) return cudaSuccess;
    const int64_t grid = tiles < sms ? tiles : sms;
    gemm_tf32x3_tc_kernel<<<(unsigned)grid, T3J_THREADS, smem, s>>>(J, status);
    J.n = 0;
    tiles = 0;
    return cudaGetLastError();
  };
  for (int i = 0; i < n; ++i) {
    const T3JobDesc& q = d[i];
    if (q.seg_rows <= 0 || q.n_seg <= 0 || q.n_out <= 0) continue;
    if (q.K % 4 || q.ldx % 4 || q.ldw % 4 || q.x_seg_stride % 4 || (uintptr_t)q.X % 16 || (uintptr_t)q.Wbig % 16 ||
        (uintptr_t)q.Wsmall % 16 || q.bias_period <= 0 || q.seg_rows > (int64_t)INT32_MAX ||
        q.n_seg > (int64_t)INT32_MAX)
      return cudaErrorInvalidValue;
    T3Job& j = J.j[J.n];
    int rb = TC_BM;  // short segments: several per tile, rb (a power of two >= 8) rows each
    while (rb > 8 && rb / 2 >= q.seg_rows) rb /= 2;
    if (!make_map_seg_f32(&j.a, q.X, q.seg_rows, q.n_seg, q.K, q.ldx,
                          q.n_seg > 1 ? q.x_seg_stride : q.seg_rows * q.ldx, rb) ||
        !make_map(&j.bb, q.Wbig, q.n_out, q.K, q.ldw ? q.ldw : q.K, TC_BN, true) ||
        !make_map(&j.bs, q.Wsmall, q.n_out, q.K, q.ldw ? q.ldw : q.K, TC_BN, true))
      return cudaErrorInvalidValue;
    j.f.bias = q.bias;
    j.f.Y = q.Y;
    j.f.seg_rows = q.seg_rows;
    j.f.n_seg = q.n_seg;
    j.f.ldy = q.ldy;
    j.f.y_seg_stride = q.y_seg_stride;
    j.f.rb = rb;
    j.f.sb = TC_BM / rb;
    j.f.rb_per_seg = (q.seg_rows + rb - 1) / rb;
    j.f.n_mblk = ((q.n_seg + j.f.sb - 1) / j.f.sb) * j.f.rb_per_seg;
    j.f.n_out = q.n_out;
    j.f.nk = (q.K + T3_BK - 1) / T3_BK;  // a ragged last K block reads zeros past K
    j.f.n_tiles_n = (q.n_out + TC_BN - 1) / TC_BN;
    j.f.bias_period = q.bias_period;
    j.f.accumulate = q.accumulate ? 1 : 0;
    tiles += ((j.f.n_mblk + T3_SUB - 1) / T3_SUB) * j.f.n_tiles_n;
    j.f.tile_end = tiles;
    if (++J.n == kT3MaxJobs) {
      e = flush();
      if (e != cudaSuccess) return e;
    }
  }
  return flush();
}

cudaError_t gemm_tf32x3_tc_seg(const float* X, int64_t seg_rows, int64_t n_seg, int64_t x_seg_stride, int K,
                               int64_t ldx, const float* Wbig, const float* Wsmall, int n_out, const float* bias,
                               int bias_period, float* Y, int64_t ldy, int64_t y_seg_stride, unsigned int* status,
                               cudaStream_t s, bool accumulate) {
  const T3JobDesc d{X, seg_rows, n_seg, x_seg_stride, K, ldx, Wbig, Wsmall, n_out, bias, bias_period, Y, ldy,
                    y_seg_stride, accumulate};
  return gemm_tf32x3_tc_jobs(&d, 1, status, s);
}

// FP32 rows [n_seg][rps] x cols, dims {cols, rps, n_seg}, box {128, rb, 32 / rb}, no swizzle
bool make_map_rows_f32(CUtensorMap* m, const void* base, int64_t rps, int64_t n_seg, int cols, int64_t pitch,
                       int64_t seg_stride, int rb) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rps, (cuuint64_t)n_seg};
  const cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)seg_stride * 4};
  const cuuint32_t box[3] = {(cuuint32_t)TC_BM, (cuuint32_t)rb, (cuuint32_t)(TN_BK / rb)};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
constexpr size_t tn_smem_bytes() {
  return 1024 + TN_TSTAGES * 2 * TN_TILE + TN_OSTAGES * 4 * TN_TILE + (2 * TN_TSTAGES + 2 * TN_OSTAGES + 4) * 8 + 16;
}

cudaError_t gemm_tn_tf32x3(const float* X, int64_t x_pitch, int64_t x_seg_stride, const float* Y, int64_t y_pitch,
                           int64_t y_seg_stride, int64_t rps, int64_t n_seg, int n_o, int n_a, float* part,
                           int64_t part_elems, int64_t* splits_out, unsigned int* status, cudaStream_t s,
                           float** colpart_out) {
  *splits_out = 0;
  if (rps <= 0 || n_seg <= 0 || n_o <= 0 || n_a <= 0) return cudaSuccess;
  if (x_pitch % 4 || y_pitch % 4 || x_seg_stride % 4 || y_seg_stride % 4 || (uintptr_t)X % 16 || (uintptr_t)Y % 16 ||
      rps > (int64_t)INT32_MAX || n_seg > (int64_t)INT32_MAX)
    return cudaErrorInvalidValue;
  int rb = TN_BK;  // short segments: several per K step
  while (rb > 1 && rb / 2 >= rps) rb /= 2;
  CUtensorMap mx, my;
  if (!make_map_rows_f32(&mx, X, rps, n_seg, n_o, x_pitch, x_seg_stride, rb) ||
      !make_map_rows_f32(&my, Y, rps, n_seg, n_a, y_pitch, y_seg_stride, rb))
    return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (int64_t)((n_o + TC_BM - 1) / TC_BM) * ((n_a + TC_BN - 1) / TC_BN);
  const int64_t ktot = ((n_seg + TN_BK / rb - 1) / (TN_BK / rb)) * ((rps + rb - 1) / rb);
  int64_t splits = (sms + tiles - 1) / tiles;  // about one work item per SM
  if (splits > ktot) splits = ktot;
  // per split: the partial tile, and with column sums one partial row of n_o
  const int64_t per_split = (int64_t)n_o * n_a + (colpart_out ? n_o : 0);
  if (splits * per_split > part_elems) splits = part_elems / per_split;
  if (splits < 1) return cudaErrorInvalidValue;
  const int64_t kps = (ktot + splits - 1) / splits;
  splits = (ktot + kps - 1) / kps;  // every split has at least one K step
  float* colpart = colpart_out ? part + splits * (int64_t)n_o * n_a : nullptr;
  const size_t smem = tn_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(gemm_tn_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t items = tiles * splits;
  const int64_t grid = items < sms ? items : sms;
  gemm_tn_tf32x3_kernel<<<(unsigned)grid, T3_THREADS, smem, s>>>(mx, my, rps, n_seg, rb, n_o, n_a, splits, kps, part,
                                                                colpart, status);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    *splits_out = splits;
    if (colpart_out) *colpart_out = colpart;
  }
  return e;
}

cudaError_t gemm_tf32x3_tc(const float* X, int64_t rows, int K, int64_t ldx, const float* Wbig, const float* Wsmall,
                           int n_out, const float* bias, int bias_period, float* Y, int64_t ldy, unsigned int* status,
                           cudaStream_t s) {
  return gemm_tf32x3_tc_seg(X, rows, 1, 0, K, ldx, Wbig, Wsmall, n_out, bias, bias_period, Y, ldy, 0, status, s,
                            false);
}

}  // namespace dq
