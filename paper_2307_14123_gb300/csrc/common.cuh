// Internal declarations shared by the CUDA translation units of libdqmc.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/dqmc.h"

namespace dq {

constexpr int kMaxElec = 64;   // n_up + n_down
constexpr int kMaxSpin = 32;   // electrons per spin channel (one warp per matrix)
constexpr int kMaxNuc = 64;

// Element offsets of the blocks of the flat parameter vector (layout in dqmc.h).
struct ParamOffsets {
  int64_t E_spin;                    // -1 with the electron-nucleus initial embedding
  int64_t W_e1, b_e1, W_e2, b_e2;    // that embedding's MLP (-1 without it)
  struct Layer {
    int64_t W_h, U[3], c[3], W1[3], b1[3], W2[3], b2[3], Y, W_g, b_g;  // U, c: -1 without edge updates
  } layer[16];
  int64_t W_o[2], b_o[2], omega[2], zeta[2], c, W_J1, b_J1, w_J2, total;
};
constexpr int kMaxLayers = 16;

ParamOffsets make_offsets(int D, int L, int K, int Q, int M, int nc_up, int nc_dn, int edge_update, int el_init);

// Edge bookkeeping.  Electron-electron pairs (i < j) are ordered by type:
// up-up pairs, down-down pairs (together: same spin), then up-down pairs
// (opposite spin); electron-nucleus edges (i, I) follow at E_ee + i*M + I.
struct Edges {
  int n_par, n_anti, n_ee, n_en, n_all;
};

}  // namespace dq

namespace dq {
// Kernel kinds for the optional per-launch timing (dq_profile_*).  The
// value-only forward (ansatz_eval, Metropolis) uses kind + kValueOffset.
enum ProfKind {
  PK_GEOMETRY = 0, PK_EDGE_HIDDEN, PK_GEMM_EDGE, PK_MESSAGES, PK_GEMM_NODE, PK_GEMM_UPDATE, PK_UPDATE,
  PK_GEMM_ORBITAL, PK_ORBITAL_DET, PK_JASTROW_SUM, PK_GEMM_JASTROW, PK_COMBINE, PK_LAYER0, PK_LAYER_FUSED,
  PK_FWD_KINDS,
  PK_ESUM = 2 * PK_FWD_KINDS, PK_PROPOSE, PK_ACCEPT, PK_LOSS_WEIGHTS, PK_BWD_COMBINE, PK_BWD_DET, PK_BWD_GEMM,
  PK_BWD_UPDATE, PK_BWD_MESSAGES, PK_BWD_EDGE, PK_BWD_REDUCE, PK_COUNT
};
constexpr int kValueOffset = PK_FWD_KINDS;
const char* prof_kind_name(int k);

struct Profiler {
  bool on = false;
  bool overflow = false;
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  std::vector<int> kinds;  // kind of record r; events 2r, 2r+1 of the pool
  void begin(int kind, cudaStream_t s) {
    if (!on) return;
    if (next + 2 > pool.size()) {
      overflow = true;
      return;
    }
    kinds.push_back(kind);
    cudaEventRecord(pool[next], s);
    next += 1;
  }
  void end(cudaStream_t s) {
    if (!on || overflow) return;
    cudaEventRecord(pool[next], s);
    next += 1;
  }
};
}  // namespace dq

namespace dq {
// Table of a grouped launch: one kernel launch over several molecules (or
// other independent problems).  Entry m owns blocks end[m-1] .. end[m] - 1 of
// the 1-D grid, which it sees as an nbx x ny grid (flattened x-major); tag
// selects a variant of the kernel body for the entry.
constexpr int kMaxGroup = 8;
template <class A>
struct Grp {
  A a[kMaxGroup];
  int64_t end[kMaxGroup];
  int64_t nbx[kMaxGroup];
  int ny[kMaxGroup];
  int tag[kMaxGroup];
  int n;
  void add(const A& x, int64_t bx, int by = 1, int t = 0) {
    a[n] = x;
    nbx[n] = bx;
    ny[n] = by;
    tag[n] = t;
    end[n] = (n > 0 ? end[n - 1] : 0) + bx * by;
    ++n;
  }
  int64_t blocks() const { return n > 0 ? end[n - 1] : 0; }
};
// Reads of a kernel's parameter block at run-time offsets are slow, so the
// table is read at compile-time offsets only: the entry search is unrolled,
// and GRP_STATIC runs a block of code once per entry index K_ (a constant)
// through a switch.  The empty asm with the index as an immediate keeps the
// compiler from merging the cases back into one run-time-indexed read.
template <class A>
__device__ __forceinline__ int grp_find(const Grp<A>& g, int64_t blk, int64_t& local) {
  int m = 0;
  int64_t start = 0;
#pragma unroll
  for (int k = 0; k + 1 < kMaxGroup; ++k)
    if (k + 1 < g.n && blk >= g.end[k]) {
      m = k + 1;
      start = g.end[k];
    }
  local = blk - start;
  return m;
}
// Entry m's block l as (x, y) of its nbx x ny grid; l < 2^31 (checked at launch).
template <class A>
__device__ __forceinline__ int64_t grp_bx(const Grp<A>& g, int m, int64_t l) {
  const int ny = g.ny[m];
  return ny == 1 ? l : (int64_t)((uint32_t)l / (uint32_t)ny);
}
template <class A>
__device__ __forceinline__ int grp_by(const Grp<A>& g, int m, int64_t l) {
  const int ny = g.ny[m];
  return ny == 1 ? 0 : (int)((uint32_t)l % (uint32_t)ny);
}
#define GRP_CASE(K, ...)            \
  case K: {                         \
    asm volatile("" ::"n"(K));      \
    constexpr int K_ = K;           \
    __VA_ARGS__                     \
  } break;
#define GRP_STATIC(m, ...)                                                                     \
  switch (m) {                                                                                 \
    GRP_CASE(0, __VA_ARGS__) GRP_CASE(1, __VA_ARGS__) GRP_CASE(2, __VA_ARGS__)                 \
    GRP_CASE(3, __VA_ARGS__) GRP_CASE(4, __VA_ARGS__) GRP_CASE(5, __VA_ARGS__)                 \
    GRP_CASE(6, __VA_ARGS__) GRP_CASE(7, __VA_ARGS__)                                          \
  }
}  // namespace dq

struct dq_handle_s {
  int device = 0;
  int precision = 0;
  int n_up = 0, n_dn = 0, N = 0, M = 0;
  int D = 0, L = 0, K = 0, Q = 0;
  double rc = 10.0, alpha = 1.0;
  int use_jastrow = 1, use_cusp = 1;
  int full_det = 0;  // 1: one N x N determinant per p (Eq. 22) instead of det A^up det A^down (Eq. 21)
  int edge_update = 0;  // 1: edge embeddings iterated between layers (Eq. 16, second case)
  int el_init = 0;      // 1: initial embeddings from electron-nucleus differences (Eq. 13, second case)
  double Vnn = 0;
  // Orbitals per determinant of spin sg's orbital network: n_sg, or N for the full determinant.
  int ncol(int sg) const { return full_det ? N : (sg ? n_dn : n_up); }
  // Side of the largest determinant matrix; the orbital row pitch is K * det_n().
  int det_n() const { return full_det ? N : (n_up > n_dn ? n_up : n_dn); }
  dq::ParamOffsets off{};
  dq::Edges edges{};
  int64_t max_chunk = 4096;
  int msg_ib = 0;  // receivers per warp task of the jet message kernel (FP32 modes: 8 or 4; 0: 8)
  int msg_kernel = 0;  // jet message kernel of the separate path: 1 general, 2 sender-tiled, 0 by size
  int layer_kernel = 0;  // jet layers: 0 fused kernel where supported, 1 the same, 2 separate kernels
  int det_warps = 4;     // warps (matrices) per CTA of the grouped determinant kernels: 4 or 2
  // device tables
  double* d_R = nullptr;   // [M][3]
  float* d_Rf = nullptr;   // [M][3]
  double* d_Z = nullptr;   // [M]
  int* d_pair_of = nullptr;  // [N][N] pair index of (i, j), -1 on the diagonal
  int* d_pair_ij = nullptr;  // [n_ee][2] (i, j) with i < j
  unsigned int* d_status = nullptr;
  unsigned long long* d_fp64_count = nullptr;  // determinant matrices that took the FP64 path
  dq::Profiler* prof = nullptr;
};

// A batch of molecules: one handle per molecule (owned), launched together.
struct dq_multi_s {
  int n = 0;
  int device = 0;
  int precision = 0;
  int rounds = 0;  // walker chunks per call; 0: automatic
  dq_handle_s* h[dq::kMaxGroup] = {};
};

namespace dq {

// Row map of a row-major matrix stored in segments:
// element offset of row r = (r / rows_per_seg) * seg_stride + (r % rows_per_seg) * ld.
struct RowMap {
  int64_t rows_per_seg;
  int64_t seg_stride;
  int64_t ld;
};

// Y[r][n] (+)= sum_k X[r][k] W[n][k] + (r % bias_period == 0 ? bias[n] : 0).
// W is [n_out][K] row-major.  K % 8 == 0; X and Y rows 16-byte aligned.
template <class T>
cudaError_t gemm_nt(const T* X, RowMap mx, const T* W, const T* bias, int bias_period, T* Y, RowMap my,
                    int64_t rows, int n_out, int K, bool accumulate, cudaStream_t s);

// BF16 tensor-core GEMM (gemm_tc.cu): Y[r][n] = X[r][:] . W[n][:] (+ bias on
// rows r % bias_period == 0); X, W BF16 K-major, Y FP32.
cudaError_t gemm_bf16_tc(const void* X, int64_t rows, int K, int64_t ldx, const void* W, int n_out, const float* bias,
                         int bias_period, float* Y, int64_t ldy, unsigned int* status, cudaStream_t s);

// FP32-accurate tensor-core GEMM (3 x TF32 split, gemm_tc.cu): X FP32 [rows][K]
// (K % 4 == 0), W pre-split by split_tf32 into TF32 big and small parts.
cudaError_t split_tf32(const float* W, float* big, float* small, int64_t n, cudaStream_t s);
cudaError_t gemm_tf32x3_tc(const float* X, int64_t rows, int K, int64_t ldx, const float* Wbig, const float* Wsmall,
                           int n_out, const float* bias, int bias_period, float* Y, int64_t ldy, unsigned int* status,
                           cudaStream_t s);
// Rows in n_seg segments of seg_rows rows (segment g starts at X + g * x_seg_stride
// and Y + g * y_seg_stride; x_seg_stride % 4 == 0); the bias goes on the rows
// whose index within the segment is a multiple of bias_period.
// accumulate: Y += X W^T instead of Y = X W^T (+ bias).
cudaError_t gemm_tf32x3_tc_seg(const float* X, int64_t seg_rows, int64_t n_seg, int64_t x_seg_stride, int K,
                               int64_t ldx, const float* Wbig, const float* Wsmall, int n_out, const float* bias,
                               int bias_period, float* Y, int64_t ldy, int64_t y_seg_stride, unsigned int* status,
                               cudaStream_t s, bool accumulate = false);
// Pseudopotentials (pseudo.cu): the coefficient set travels as a kernel parameter.
constexpr int kMaxPP = 8, kMaxPPChan = 5, kMaxPPTerms = 4;  // nuclei, channels (V, W_0..W_3), Gaussian terms
struct PPSet {
  int n;                      // pseudopotentials
  int nucleus[kMaxPP];
  int lmax[kMaxPP];
  int n_terms[kMaxPP];
  double c[kMaxPP * kMaxPPChan * kMaxPPTerms][3];  // [q][channel][term]: beta, n, alpha
};
template <class T>
cudaError_t pp_displace(const T* r, const double* Rn, const T* rot, int64_t B, int N, const PPSet& pp, T* configs,
                        cudaStream_t s);
template <class T>
cudaError_t pp_combine(const T* r, const double* Rn, const T* rot, const T* logabs, const int8_t* sign, const T* la_c,
                       const int8_t* sg_c, int64_t B, int N, const PPSet& pp, T* v_loc, T* v_nl, cudaStream_t s);
// Natural-gradient direction (natgrad.cu): workspace bytes and the computation for B
// walkers' gradients G [B][P] and weights w [B].
size_t natgrad_workspace(int64_t B, int64_t P);
cudaError_t natgrad_run(const float* G, const float* w, int64_t B, int64_t P, double lam, int max_iter, double tol,
                        float* delta, double* stats, unsigned char* ws, unsigned int* status, cudaStream_t s);
// Parameter update theta -= lr s delta with s = min(1, max_norm / (lr ||delta||)); stats
// (device double[2]): ||delta||, s.  Workspace: param_update_workspace() bytes.
size_t param_update_workspace();
template <class T>
cudaError_t param_update_run(T* theta, const T* delta, int64_t P, double lr, double max_norm, double* stats,
                             unsigned char* ws, cudaStream_t s);
// A list of such GEMMs in one persistent launch (tiles of all jobs share the
// grid); at most 16 per launch (more are split over launches).
struct T3JobDesc {
  const float* X;
  int64_t seg_rows, n_seg, x_seg_stride;
  int K;
  int64_t ldx;
  const float *Wbig, *Wsmall;
  int n_out;
  const float* bias;
  int bias_period;
  float* Y;
  int64_t ldy, y_seg_stride;
  bool accumulate;
  int64_t ldw = 0;  // row pitch of Wbig / Wsmall in elements (0: K)
};
cudaError_t gemm_tf32x3_tc_jobs(const T3JobDesc* jobs, int n, unsigned int* status, cudaStream_t s);
// TF32 high / low parts of the transpose of W [rows][cols] (for products X W).
cudaError_t split_tf32_t(const float* W, int rows, int cols, float* big, float* small, cudaStream_t s);
// Row reduction part[split][o][a] = sum_r X[r][o] Y[r][a] on the tensor cores (3 x TF32); rows in n_seg
// segments of rps rows (row pitch, segment stride in elements; multiples of 4, 16-byte aligned bases).
// The split count (every split non-empty, splits * n_o * n_a <= part_elems) is returned in splits_out.
// colpart_out non-null: the column sums of X per split as well (colpart[split][o], placed after the
// partial tiles in part, counted in part_elems), their address returned in *colpart_out.
cudaError_t gemm_tn_tf32x3(const float* X, int64_t x_pitch, int64_t x_seg_stride, const float* Y, int64_t y_pitch,
                           int64_t y_seg_stride, int64_t rps, int64_t n_seg, int n_o, int n_a, float* part,
                           int64_t part_elems, int64_t* splits_out, unsigned int* status, cudaStream_t s,
                           float** colpart_out = nullptr);

// ---- forward kernels (forward.cu) ------------------------------------------
// Sizes of one chunk of Bc walkers; C = channels (1 value-only, 3N+2 with jets).
struct FwdDims {
  int64_t Bc;
  int N, n_up, n_dn, M, D, K, Q, C;
};

template <class T>
struct FwdBuffers {
  T* geo;    // [Bc][E][4]          distance and unit vector of every edge
  T* rbf;    // [Bc][E][3][Q]       Gaussian features and d/dd, d2/dd2
  T* eh;     // [Bc][E][3][D]       edge hidden layer jets (value, d/dd, d2/dd2)
  T* ew;     // [Bc][E][3][D]       edge filter jets
  T* F;      // [Bc][N][C][D]       embeddings with jets
  T* Z;      // [Bc][N][C][D]       W_h f, then the update pre-activation
  T* msg;    // [Bc][N][C][3D]      messages [par | anti | nuc]
  T* phi;    // [Bc][N][C][K nmax]  orbital head output
  double* det;  // [Bc][2][K][3N+3] sign, log|det|, grad, laplacian
  T* js;     // [Bc][C][D]          sum_i f_i
  T* jh;     // [Bc][C][D]          W_J1 (sum_i f_i) + b_J1
  T* z0;     // [2][D]              W_h^0 E_spin
  // BF16 mode only (nullptr otherwise): GEMM inputs of the embedding layers
  void* msg_bf;  // [Bc][N][C][3D]  messages, BF16 (replaces msg)
  void* F_bf;    // [Bc][N][C][D]   BF16 copy of the embeddings
};

// Grouped sampler and reduction launches (mcmc.cu), one entry per molecule.
template <class T>
cudaError_t launch_propose_group(const dq_handle_s* const* hs, int n, const int64_t* B, const T* const* r,
                                 T* const* r_prop, double step, uint64_t seed, uint64_t t, const uint64_t* t_base,
                                 cudaStream_t s);
template <class T>
cudaError_t launch_accept_group(const dq_handle_s* const* hs, int n, const int64_t* B, T* const* r, T* const* logabs,
                                const T* const* r_prop, const T* const* la_prop, const int8_t* const* sign_prop,
                                uint64_t seed, uint64_t t, const uint64_t* t_base, unsigned long long* const* n_acc,
                                cudaStream_t s, T* e_loc = nullptr, const T* e_prop = nullptr);
template <class T>
cudaError_t launch_esum_group(int n, const T* const* e, const int64_t* B, double* const* out2,
                              unsigned int* const* status, cudaStream_t s);
template <class T>
cudaError_t launch_loss_weights_group(int n, const T* const* e, const int64_t* B, double k, T* const* w,
                                      double* const* stats, double* const* scratch, cudaStream_t s, int soft = 0);

// One molecule of a grouped launch: its handle, chunk dimensions, parameters and buffers.
template <class T>
struct MolFwd {
  const dq_handle_s* h;
  FwdDims d;
  const T* params;
  FwdBuffers<T> b;
};
template <class T>
cudaError_t launch_geometry_group(const MolFwd<T>* m, int n, const T* const* r, cudaStream_t s);
template <class T>
cudaError_t launch_edge_hidden_group(const MolFwd<T>* m, int n, int layer, cudaStream_t s);
// Iterated edge embeddings of layer `layer` >= 1 (nothing for handles without them): dst = u(src).
template <class T>
cudaError_t launch_edge_update_group(const MolFwd<T>* m, int n, int layer, const T* const* src, T* const* dst,
                                     cudaStream_t s);
template <class T>
cudaError_t launch_edge_update(const dq_handle_s& h, const FwdDims& d, const T* params, int layer, const T* src,
                               T* dst, cudaStream_t s);
// Initial embeddings from the electron-nucleus difference vectors (Eq. 13, second case) for a
// chunk of d.Bc walkers at r: F[Bc][N][C][D] with its jets (C > 1) or values (C = 1); Fbf
// (nullable) a BF16 copy; H0 [Bc N][D] and X0 [Bc N][3M] (nullable) keep the hidden layer
// and the difference vectors for the reverse pass.
template <class T>
cudaError_t launch_el_init(const dq_handle_s& h, const FwdDims& d, const T* params, const T* r, T* F, void* Fbf, T* H0,
                           T* X0, cudaStream_t s);
template <class T>
cudaError_t launch_layer0_node_group(const MolFwd<T>* m, int n, cudaStream_t s);
template <class T>
cudaError_t launch_messages_group(const MolFwd<T>* m, int n, int layer, bool z_const, cudaStream_t s);
template <class T>
cudaError_t launch_update_group(const MolFwd<T>* m, int n, bool from_spin, cudaStream_t s);

// The message and update-map part of one jets layer (layer_fused.cu): the electron-electron
// messages (Eq. 17) as the A operand of the update map W_g on the tensor cores (three TF32
// products; BF16 operands when wg_bf, the BF16 copy of W_g, is given), so that they never reach
// memory; the electron-nucleus messages, non-zero on five channels per electron, go through W_g's
// third block apart (3 x TF32) and are added after.  Writes the pre-activations u = W_g m + b_g
// into Z in place (the tanh update of Eq. 18 follows as in the separate path).  mn: workspace of
// Bc N 11 D floats.  FP32 and BF16 modes, D = 128, N <= 16 with at most 8 electrons per spin and
// 8 nuclei.
bool layer_fused_supported(const dq_handle_s& h);
// Jet messages of molecules past the fused layer kernel (messages_large.cu): FP32 modes, node
// channels from the node map (not the spin-embedding constants), 3 N + 2 channels, D a multiple
// of 32, N <= 48 with at most 24 electrons per spin.  Writes all three message slots of msg
// ([Bc][N][C][3D], FP32, or BF16 when bf16_out).
bool messages_large_supported(const dq_handle_s& h, const FwdDims& d);
cudaError_t launch_messages_large(const dq_handle_s& h, const FwdDims& d, const float* params, int l,
                                  const float* Z, const float* ew, const float* geo, void* msg, bool bf16_out,
                                  cudaStream_t s);
cudaError_t launch_layer_fused(const dq_handle_s& h, const FwdDims& d, const float* params, int l, bool z_const,
                               float* Z, const float* z0, const float* ew, const float* geo, float* mn,
                               const float* wg_hi, const float* wg_lo, const void* wg_bf, cudaStream_t s);
template <class T>
cudaError_t launch_orbital_det_group(const MolFwd<T>* m, int n, cudaStream_t s);
template <class T>
cudaError_t launch_jastrow_sum_group(const MolFwd<T>* m, int n, cudaStream_t s);
template <class T>
cudaError_t launch_combine_group(const MolFwd<T>* m, int n, T* const* logabs, int8_t* const* sign, T* const* e_loc,
                                 T* const* grad, cudaStream_t s);

template <class T>
cudaError_t launch_geometry(const dq_handle_s& h, const FwdDims& d, const T* r, FwdBuffers<T> b, cudaStream_t s);
template <class T>
cudaError_t launch_edge_hidden(const dq_handle_s& h, const FwdDims& d, const T* params, int layer,
                               FwdBuffers<T> b, cudaStream_t s);
template <class T>
cudaError_t launch_layer0_node(const dq_handle_s& h, const FwdDims& d, const T* params, FwdBuffers<T> b,
                               cudaStream_t s);
template <class T>
cudaError_t launch_messages(const dq_handle_s& h, const FwdDims& d, const T* params, int layer, bool z_const,
                            FwdBuffers<T> b, cudaStream_t s);
template <class T>
cudaError_t launch_update(const dq_handle_s& h, const FwdDims& d, const T* params, bool from_spin,
                          FwdBuffers<T> b, cudaStream_t s);
template <class T>
cudaError_t launch_update_io(const dq_handle_s& h, const FwdDims& d, const T* params, bool from_spin, const T* P,
                             const T* Fin, T* Fout, cudaStream_t s, void* Fbf = nullptr);
// dst[k] = bf16(src[k]), k < n.
cudaError_t launch_to_bf16(const float* src, void* dst, int64_t n, cudaStream_t s);
template <class T>
cudaError_t launch_orbital_det(const dq_handle_s& h, const FwdDims& d, const T* params, FwdBuffers<T> b,
                               cudaStream_t s);
template <class T>
cudaError_t launch_jastrow_sum(const dq_handle_s& h, const FwdDims& d, FwdBuffers<T> b, cudaStream_t s);
template <class T>
cudaError_t launch_combine(const dq_handle_s& h, const FwdDims& d, const T* params, FwdBuffers<T> b,
                           T* logabs, int8_t* sign, T* e_loc, cudaStream_t s, T* grad = nullptr);

// ---- sampler, reductions, loss weights (mcmc.cu) ---------------------------
// Step t of the Philox counter: t, plus *t_base when t_base (device) is non-null.
template <class T>
cudaError_t launch_propose(const dq_handle_s& h, int64_t B, const T* r, T* r_prop, double step, uint64_t seed,
                           uint64_t t, const uint64_t* t_base, cudaStream_t s);
template <class T>
cudaError_t launch_accept(const dq_handle_s& h, int64_t B, T* r, T* logabs, const T* r_prop,
                          const T* logabs_prop, const int8_t* sign_prop, uint64_t seed, uint64_t t,
                          const uint64_t* t_base, unsigned long long* n_acc, cudaStream_t s, T* e_loc = nullptr,
                          const T* e_prop = nullptr);
// *c += n on the device (advances a device-resident step counter).
cudaError_t launch_advance_counter(uint64_t* c, uint64_t n, cudaStream_t s);
// Langevin (MALA) proposal and acceptance; g: d log|psi| / d r at r, g_prop at r_prop.
template <class T>
cudaError_t launch_mala_propose(const dq_handle_s& h, int64_t B, const T* r, const T* g, T* r_prop, T* xi,
                                double tau, uint64_t seed, uint64_t t, const uint64_t* t_base, cudaStream_t s);
template <class T>
cudaError_t launch_mala_accept(const dq_handle_s& h, int64_t B, T* r, T* logabs, T* g, const T* r_prop,
                               const T* la_prop, const int8_t* sign_prop, const T* g_prop, const T* xi, T* e_loc,
                               const T* e_prop, double tau, uint64_t seed, uint64_t t, const uint64_t* t_base,
                               unsigned long long* n_acc, cudaStream_t s);
template <class T>
cudaError_t launch_esum(const T* e, int64_t B, double* out2, unsigned int* status, cudaStream_t s);
template <class T>
cudaError_t launch_loss_weights(const T* e, int64_t B, double k, T* w, double* stats, double* scratch,
                                cudaStream_t s, int soft = 0);

}  // namespace dq
