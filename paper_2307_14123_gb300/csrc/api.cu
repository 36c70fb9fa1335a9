// C ABI of libdqmc (declarations and contracts in include/dqmc.h).
//
// Host-side orchestration only: argument checks, the flat parameter layout,
// edge tables, workspace carving, and the stream-ordered launch sequence of
// the hot path.  Every arithmetic step runs in the CUDA kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <initializer_list>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "backward.cuh"
#include "common.cuh"

namespace dq {

// nc_up, nc_dn: orbitals per determinant of the spin-up and spin-down networks;
// edge_update: the edge-embedding maps U, c of layers l >= 1 precede each type's filter.
// el_init: the initial-embedding MLP W_e1[D][3M], b_e1[D], W_e2[D][D], b_e2[D] in place of E_spin.
ParamOffsets make_offsets(int D, int L, int K, int Q, int M, int nc_up, int nc_dn, int edge_update, int el_init) {
  ParamOffsets o{};
  int64_t p = 0;
  o.E_spin = o.W_e1 = o.b_e1 = o.W_e2 = o.b_e2 = -1;
  if (el_init) {
    o.W_e1 = p;
    p += (int64_t)D * 3 * M;
    o.b_e1 = p;
    p += D;
    o.W_e2 = p;
    p += (int64_t)D * D;
    o.b_e2 = p;
    p += D;
  } else {
    o.E_spin = p;
    p += 2 * (int64_t)D;
  }
  for (int l = 0; l < L; ++l) {
    auto& y = o.layer[l];
    y.W_h = p;
    p += (int64_t)D * D;
    for (int t = 0; t < 3; ++t) {
      y.U[t] = y.c[t] = -1;
      if (edge_update && l > 0) {
        y.U[t] = p;
        p += (int64_t)Q * Q;
        y.c[t] = p;
        p += Q;
      }
      y.W1[t] = p;
      p += (int64_t)D * Q;
      y.b1[t] = p;
      p += D;
      y.W2[t] = p;
      p += (int64_t)D * D;
      y.b2[t] = p;
      p += D;
    }
    y.Y = p;
    p += (int64_t)M * D;
    y.W_g = p;
    p += (int64_t)3 * D * D;
    y.b_g = p;
    p += D;
  }
  const int ns[2] = {nc_up, nc_dn};
  for (int s = 0; s < 2; ++s) {
    o.W_o[s] = p;
    p += (int64_t)K * ns[s] * D;
    o.b_o[s] = p;
    p += (int64_t)K * ns[s];
    o.omega[s] = p;
    p += (int64_t)K * ns[s] * M;
    o.zeta[s] = p;
    p += (int64_t)K * ns[s] * M;
  }
  o.c = p;
  p += K;
  o.W_J1 = p;
  p += (int64_t)D * D;
  o.b_J1 = p;
  p += D;
  o.w_J2 = p;
  p += D;
  o.total = p;
  return o;
}

const char* prof_kind_name(int k) {
  static const char* fwd[PK_FWD_KINDS] = {"geometry", "edge_hidden", "gemm_edge", "messages", "gemm_node",
                                          "gemm_update", "update", "gemm_orbital", "orbital_det", "jastrow_sum",
                                          "gemm_jastrow", "combine", "layer0_node", "layer_fused"};
  static const char* fwd_jet[PK_FWD_KINDS];
  static const char* other[PK_COUNT - 2 * PK_FWD_KINDS] = {"esum", "propose", "accept", "loss_weights",
                                                           "bwd_combine", "bwd_det", "bwd_gemm", "bwd_update",
                                                           "bwd_messages", "bwd_edge", "bwd_reduce"};
  static char names[PK_COUNT][40];
  static bool init = false;
  if (!init) {
    for (int i = 0; i < PK_FWD_KINDS; ++i) {
      snprintf(names[i], 40, "jet.%s", fwd[i]);
      snprintf(names[PK_FWD_KINDS + i], 40, "val.%s", fwd[i]);
    }
    for (int i = 2 * PK_FWD_KINDS; i < PK_COUNT; ++i) snprintf(names[i], 40, "%s", other[i - 2 * PK_FWD_KINDS]);
    init = true;
  }
  (void)fwd_jet;
  return (k >= 0 && k < PK_COUNT) ? names[k] : "unknown";
}

namespace {

constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Sub-buffer offsets (bytes) of the forward workspace for a chunk of Bc walkers.
struct FwdPlan {
  size_t geo, rbf, eh, ew, F, Z, msg, phi, det, js, jh, z0, msg_bf, F_bf, W_bf, W_t3, total;
};

// FP32 modes: the FP32 GEMMs (edge filters, node and update maps, orbitals)
// run on the tensor cores as 3 x TF32 products when the width allows the
// 128-byte TMA rows (D % 32 == 0); in BF16 mode the node and update maps take
// the BF16 GEMM instead.
inline bool use_tf32x3(const dq_handle_s& h) { return h.precision != DQ_FP64 && h.D % 32 == 0; }
// Jet layers through the fused message / update-map / update kernel (layer_fused.cu).
inline bool use_fused(const dq_handle_s& h, bool jets) {
  return jets && h.layer_kernel != 2 && use_tf32x3(h) && layer_fused_supported(h);
}
constexpr int kT3PerLayer = 14;  // D x D blocks per layer: W_g 2 x 3, W_h 2, W2 2 x 3
// TF32 splits: the layers' blocks, then W_o of both spins (high, low; K * nmax x D
// each), then the Jastrow map W_J1 (high, low; D x D)
inline int64_t t3_weight_floats(const dq_handle_s& h) {
  const int64_t nmax = h.det_n();
  return (int64_t)h.L * kT3PerLayer * h.D * h.D + 4 * h.K * nmax * h.D + 2 * (int64_t)h.D * h.D;
}
// Views of the split weights; part 0 = TF32 high, 1 = low.
struct T3Weights {
  float* base;
  int64_t DD, WoD;
  int L;
  // layer l: W_g high [3DD], W_g low [3DD], W_h high [DD], W_h low [DD], W2[t] high / low [DD]
  float* wg(int l, int part) const { return base + (int64_t)l * kT3PerLayer * DD + part * 3 * DD; }
  float* wh(int l, int part) const { return base + (int64_t)l * kT3PerLayer * DD + 6 * DD + part * DD; }
  float* w2(int l, int t, int part) const { return base + (int64_t)l * kT3PerLayer * DD + (8 + 2 * t + part) * DD; }
  float* wo(int sg, int part) const { return base + (int64_t)L * kT3PerLayer * DD + (2 * sg + part) * WoD; }
  float* wj(int part) const { return base + (int64_t)L * kT3PerLayer * DD + 4 * WoD + part * DD; }
};
inline T3Weights t3_weights(const dq_handle_s& h, void* base) {
  return T3Weights{static_cast<float*>(base), (int64_t)h.D * h.D, (int64_t)h.K * h.det_n() * h.D,
                   h.L};
}
// Splits every weight matrix that runs on the 3 x TF32 GEMM (once per call).
cudaError_t split_t3_weights(const dq_handle_s& h, const float* params, const T3Weights& w, cudaStream_t s) {
  for (int l = 0; l < h.L; ++l) {
    cudaError_t e = split_tf32(params + h.off.layer[l].W_g, w.wg(l, 0), w.wg(l, 1), 3 * w.DD, s);
    if (e == cudaSuccess) e = split_tf32(params + h.off.layer[l].W_h, w.wh(l, 0), w.wh(l, 1), w.DD, s);
    for (int t = 0; t < 3 && e == cudaSuccess; ++t)
      e = split_tf32(params + h.off.layer[l].W2[t], w.w2(l, t, 0), w.w2(l, t, 1), w.DD, s);
    if (e != cudaSuccess) return e;
  }
  const int nsp[2] = {h.n_up, h.n_dn};
  for (int sg = 0; sg < 2; ++sg) {
    if (nsp[sg] == 0) continue;
    const cudaError_t e = split_tf32(params + h.off.W_o[sg], w.wo(sg, 0), w.wo(sg, 1), (int64_t)h.K * h.ncol(sg) * h.D, s);
    if (e != cudaSuccess) return e;
  }
  if (h.use_jastrow) return split_tf32(params + h.off.W_J1, w.wj(0), w.wj(1), w.DD, s);
  return cudaSuccess;
}

FwdPlan plan_forward(const dq_handle_s& h, int64_t Bc, bool jets, size_t elem) {
  const int64_t E = h.edges.n_all, N = h.N, D = h.D, K = h.K;
  const int64_t ej = jets ? 3 : 1, C = jets ? 3 * N + 2 : 1;
  const int64_t nmax = h.det_n();
  FwdPlan p{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += align_up(bytes);
    return at;
  };
  p.geo = take(Bc * E * 4 * elem);
  p.rbf = take(Bc * E * ej * h.Q * elem);
  p.eh = take(Bc * E * ej * D * elem);
  p.ew = take(Bc * E * ej * D * elem);
  const bool bf = h.precision == DQ_BF16_MIXED;
  p.F = take(Bc * N * C * D * elem);
  p.Z = take(Bc * N * C * D * elem);
  // messages; with the fused layer kernel (both FP32 modes) only the electron-nucleus messages of
  // five channels and their update-map products
  const bool fused = use_fused(h, jets);
  p.msg = take(fused ? Bc * N * 11 * D * elem : bf ? 0 : Bc * N * C * 3 * D * elem);
  p.phi = take(Bc * N * C * K * nmax * elem);
  p.det = take(Bc * 2 * K * (3 * N + 3) * sizeof(double));
  p.js = take(Bc * C * D * elem);
  p.jh = take(Bc * C * D * elem);
  p.z0 = take(2 * D * elem);
  // BF16 mode: messages (unless fused) and a copy of the embeddings in BF16, BF16 weights
  p.msg_bf = take(bf && !fused ? Bc * N * C * 3 * D * 2 : 0);
  p.F_bf = take(bf ? Bc * N * C * D * 2 : 0);
  p.W_bf = take(bf ? (size_t)h.L * 4 * D * D * 2 : 0);
  // FP32 mode: TF32 high and low parts of W_g, W_h and the three W2 of every layer
  p.W_t3 = take(use_tf32x3(h) ? t3_weight_floats(h) * 4 : 0);
  p.total = o;
  return p;
}

struct McmcPlan {
  size_t r_prop, la_prop, sign_prop, fwd, total;
};
// Langevin sampler: proposals, their log|psi|, sign, gradient and normals, the
// local energies the jet forward also produces, then the jet forward's workspace.
struct MalaPlan {
  size_t r_prop, la_prop, sign_prop, g_prop, xi, e_prop, fwd, total;
};
MalaPlan plan_mala(const dq_handle_s& h, int64_t B, size_t elem) {
  MalaPlan p{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += align_up(bytes);
    return at;
  };
  const size_t n3 = (size_t)B * 3 * h.N * elem;
  p.r_prop = take(n3);
  p.la_prop = take((size_t)B * elem);
  p.sign_prop = take((size_t)B);
  p.g_prop = take(n3);
  p.xi = take(n3);
  p.e_prop = take((size_t)B * elem);
  p.fwd = o;
  o += plan_forward(h, std::min<int64_t>(B, h.max_chunk), true, elem).total;
  p.total = o;
  return p;
}

McmcPlan plan_mcmc(const dq_handle_s& h, int64_t B, size_t elem) {
  McmcPlan p{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += align_up(bytes);
    return at;
  };
  p.r_prop = take((size_t)B * 3 * h.N * elem);
  p.la_prop = take((size_t)B * elem);
  p.sign_prop = take((size_t)B);
  p.fwd = o;
  o += plan_forward(h, std::min<int64_t>(B, h.max_chunk), false, elem).total;
  p.total = o;
  return p;
}

size_t loss_scratch_bytes(int64_t B) {
  int64_t Bp = 1;
  while (Bp < B) Bp <<= 1;
  return align_up((size_t)Bp * sizeof(double));
}

inline size_t elem_size(const dq_handle_s& h) { return h.precision == DQ_FP64 ? 8 : 4; }

#define DQ_CU(x)                                \
  do {                                          \
    if ((x) != cudaSuccess) return DQ_ERR_CUDA; \
  } while (0)

inline bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Launch with optional event timing on the launching stream.
#define DQ_LAUNCH(hh, kind, expr)                        \
  do {                                                  \
    if ((hh).prof) (hh).prof->begin((kind), s);         \
    const cudaError_t e_ = (expr);                      \
    if ((hh).prof) (hh).prof->end(s);                   \
    if (e_ != cudaSuccess) return DQ_ERR_CUDA;          \
  } while (0)

template <class T>
dq_status run_forward(const dq_handle_s& h, const T* params, const T* r, int64_t B, bool jets, T* logabs,
                      int8_t* sign, T* e_loc, unsigned char* ws, size_t ws_bytes, cudaStream_t s,
                      T* grad = nullptr) {
  const int64_t Bmax = std::min<int64_t>(B, h.max_chunk);
  const FwdPlan plan = plan_forward(h, Bmax, jets, sizeof(T));
  if (ws == nullptr || ws_bytes < plan.total || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  FwdBuffers<T> bf;
  bf.geo = reinterpret_cast<T*>(ws + plan.geo);
  bf.rbf = reinterpret_cast<T*>(ws + plan.rbf);
  bf.eh = reinterpret_cast<T*>(ws + plan.eh);
  bf.ew = reinterpret_cast<T*>(ws + plan.ew);
  bf.F = reinterpret_cast<T*>(ws + plan.F);
  bf.Z = reinterpret_cast<T*>(ws + plan.Z);
  bf.msg = reinterpret_cast<T*>(ws + plan.msg);
  bf.phi = reinterpret_cast<T*>(ws + plan.phi);
  bf.det = reinterpret_cast<double*>(ws + plan.det);
  bf.js = reinterpret_cast<T*>(ws + plan.js);
  bf.jh = reinterpret_cast<T*>(ws + plan.jh);
  bf.z0 = reinterpret_cast<T*>(ws + plan.z0);
  bf.msg_bf = nullptr;
  bf.F_bf = nullptr;
  // BF16 mode: the update and node maps run on the tensor cores (gemm_tc.cu)
  const bool use_tc = sizeof(T) == 4 && h.precision == DQ_BF16_MIXED;
  const bool use_t3 = sizeof(T) == 4 && use_tf32x3(h);
  const T3Weights w3 = t3_weights(h, ws + plan.W_t3);
  if (use_t3) {
    if constexpr (sizeof(T) == 4) DQ_CU(split_t3_weights(h, params, w3, s));
  }
  auto wg_t3 = [&](int l, int part) { return w3.wg(l, part); };
  auto wh_t3 = [&](int l, int part) { return w3.wh(l, part); };
  auto w2_t3 = [&](int l, int t, int part) { return w3.w2(l, t, part); };
  auto wo_t3 = [&](int sg, int part) { return w3.wo(sg, part); };
  unsigned char* W_bf = ws + plan.W_bf;
  auto wg_bf = [&](int l) { return W_bf + (size_t)l * 4 * h.D * h.D * 2; };
  auto wh_bf = [&](int l) { return wg_bf(l) + (size_t)3 * h.D * h.D * 2; };
  if (use_tc) {
    bf.msg_bf = ws + plan.msg_bf;
    bf.F_bf = ws + plan.F_bf;
    if constexpr (sizeof(T) == 4) {
      for (int l = 0; l < h.L; ++l) {
        DQ_CU(launch_to_bf16(params + h.off.layer[l].W_g, wg_bf(l), (int64_t)3 * h.D * h.D, s));
        DQ_CU(launch_to_bf16(params + h.off.layer[l].W_h, wh_bf(l), (int64_t)h.D * h.D, s));
      }
    }
  }

  const int N = h.N, D = h.D, K = h.K;
  const int C = jets ? 3 * N + 2 : 1;
  const int ej = jets ? 3 : 1;
  const int E = h.edges.n_all;
  const int Wo = K * h.det_n();
  const int kb = jets ? 0 : kValueOffset;
  if (!h.el_init)
    DQ_LAUNCH(h, kb + PK_LAYER0, launch_layer0_node<T>(h, FwdDims{Bmax, N, h.n_up, h.n_dn, h.M, D, K, h.Q, C}, params, bf, s));
  for (int64_t b0 = 0; b0 < B; b0 += Bmax) {
    const int64_t nb = std::min<int64_t>(Bmax, B - b0);
    const FwdDims d{nb, N, h.n_up, h.n_dn, h.M, D, K, h.Q, C};
    DQ_LAUNCH(h, kb + PK_GEOMETRY, launch_geometry<T>(h, d, r + b0 * N * 3, bf, s));
    // embeddings of the electron-nucleus difference vectors (Eq. 13, second case): layer 0 then
    // takes the general path below instead of the spin-embedding shortcut
    if (h.el_init)
      DQ_LAUNCH(h, kb + PK_LAYER0, launch_el_init<T>(h, d, params, r + b0 * N * 3, bf.F, use_tc ? bf.F_bf : nullptr,
                                                    nullptr, nullptr, s));
    for (int l = 0; l < h.L; ++l) {
      const auto& y = h.off.layer[l];
      if (h.edge_update && l > 0)  // edge embeddings of layer l, in place (Eq. 16, second case)
        DQ_LAUNCH(h, kb + PK_EDGE_HIDDEN, launch_edge_update<T>(h, d, params, l, bf.rbf, bf.rbf, s));
      DQ_LAUNCH(h, kb + PK_EDGE_HIDDEN, launch_edge_hidden<T>(h, d, params, l, bf, s));
      const int e0[3] = {0, h.edges.n_par, h.edges.n_ee};
      const int ng[3] = {h.edges.n_par, h.edges.n_anti, h.edges.n_en};
      if (use_t3) {  // the three edge types' filters in one launch
        T3JobDesc jd[3];
        const int64_t seg = (int64_t)E * ej * D;
        for (int t = 0; t < 3; ++t)
          jd[t] = T3JobDesc{reinterpret_cast<const float*>(bf.eh) + (int64_t)e0[t] * ej * D, (int64_t)ng[t] * ej, nb,
                            seg, D, D, w2_t3(l, t, 0), w2_t3(l, t, 1), D,
                            reinterpret_cast<const float*>(params + y.b2[t]), ej,
                            reinterpret_cast<float*>(bf.ew) + (int64_t)e0[t] * ej * D, D, seg, false};
        DQ_LAUNCH(h, kb + PK_GEMM_EDGE, gemm_tf32x3_tc_jobs(jd, 3, h.d_status, s));
      }
      for (int t = 0; t < 3 && !use_t3; ++t) {
        if (ng[t] == 0) continue;
        const RowMap m{(int64_t)ng[t] * ej, (int64_t)E * ej * D, D};
        {
          DQ_LAUNCH(h, kb + PK_GEMM_EDGE, gemm_nt<T>(bf.eh + (int64_t)e0[t] * ej * D, m, params + y.W2[t],
                                                     params + y.b2[t], ej, bf.ew + (int64_t)e0[t] * ej * D, m,
                                                     nb * ng[t] * ej, D, D, false, s));
        }
      }
      const RowMap node{(int64_t)N * C, (int64_t)N * C * D, D};
      const int64_t rows = nb * N * C;
      if (use_fused(h, jets)) {  // messages, update map and update in one kernel
        const bool z_const = l == 0 && !h.el_init;
        // the node map on 3 x TF32 in both modes: the BF16 GEMM gains nothing at K = D once the
        // update kernel has to write a BF16 copy of the embeddings for it
        if (!z_const)
          DQ_LAUNCH(h, kb + PK_GEMM_NODE, gemm_tf32x3_tc(reinterpret_cast<const float*>(bf.F), rows, D, D, wh_t3(l, 0),
                                                         wh_t3(l, 1), D, nullptr, 1, reinterpret_cast<float*>(bf.Z), D,
                                                         h.d_status, s));
        // BF16 mode: the electron-electron messages meet W_g as BF16 operands (the electron-nucleus
        // part stays on the 3 x TF32 GEMM)
        if constexpr (sizeof(T) == 4)
          DQ_LAUNCH(h, kb + PK_LAYER_FUSED,
                    launch_layer_fused(h, d, params, l, z_const, bf.Z, bf.z0, bf.ew, bf.geo, bf.msg, wg_t3(l, 0),
                                       wg_t3(l, 1), use_tc ? wg_bf(l) : nullptr, s));
        FwdBuffers<T> bu = bf;
        bu.F_bf = nullptr;  // no BF16 copy of the embeddings: nothing on this path reads one
        DQ_LAUNCH(h, kb + PK_UPDATE, launch_update<T>(h, d, params, z_const, bu, s));
        continue;
      }
      if (l == 0 && !h.el_init) {
        DQ_LAUNCH(h, kb + PK_MESSAGES, launch_messages<T>(h, d, params, l, true, bf, s));
      } else {
        if (use_tc) {
          DQ_LAUNCH(h, kb + PK_GEMM_NODE, gemm_bf16_tc(bf.F_bf, rows, D, D, wh_bf(l), D, nullptr, 1,
                                                       reinterpret_cast<float*>(bf.Z), D, h.d_status, s));
        } else if (use_t3) {
          DQ_LAUNCH(h, kb + PK_GEMM_NODE, gemm_tf32x3_tc(reinterpret_cast<const float*>(bf.F), rows, D, D, wh_t3(l, 0),
                                                         wh_t3(l, 1), D, nullptr, 1, reinterpret_cast<float*>(bf.Z), D,
                                                         h.d_status, s));
        } else {
          DQ_LAUNCH(h, kb + PK_GEMM_NODE, gemm_nt<T>(bf.F, node, params + y.W_h, nullptr, 1, bf.Z, node, rows, D, D,
                                                     false, s));
        }
        DQ_LAUNCH(h, kb + PK_MESSAGES, launch_messages<T>(h, d, params, l, false, bf, s));
      }
      const RowMap mrow{(int64_t)N * C, (int64_t)N * C * 3 * D, 3 * D};
      if (use_tc) {
        DQ_LAUNCH(h, kb + PK_GEMM_UPDATE, gemm_bf16_tc(bf.msg_bf, rows, 3 * D, 3 * D, wg_bf(l), D,
                                                       reinterpret_cast<const float*>(params + y.b_g), C,
                                                       reinterpret_cast<float*>(bf.Z), D, h.d_status, s));
      } else if (use_t3) {
        DQ_LAUNCH(h, kb + PK_GEMM_UPDATE, gemm_tf32x3_tc(reinterpret_cast<const float*>(bf.msg), rows, 3 * D, 3 * D,
                                                         wg_t3(l, 0), wg_t3(l, 1), D,
                                                         reinterpret_cast<const float*>(params + y.b_g), C,
                                                         reinterpret_cast<float*>(bf.Z), D, h.d_status, s));
      } else {
        DQ_LAUNCH(h, kb + PK_GEMM_UPDATE, gemm_nt<T>(bf.msg, mrow, params + y.W_g, params + y.b_g, C, bf.Z, node, rows,
                                                     D, 3 * D, false, s));
      }
      DQ_LAUNCH(h, kb + PK_UPDATE, launch_update<T>(h, d, params, l == 0 && !h.el_init, bf, s));
    }
    const int ns[2] = {h.n_up, h.n_dn}, i0[2] = {0, h.n_up};
    if (use_t3) {  // both spins' orbitals in one launch
      T3JobDesc jd[2];
      for (int sg = 0; sg < 2; ++sg)
        jd[sg] = T3JobDesc{reinterpret_cast<const float*>(bf.F) + (int64_t)i0[sg] * C * D, (int64_t)ns[sg] * C, nb,
                           (int64_t)N * C * D, D, D, wo_t3(sg, 0), wo_t3(sg, 1), K * h.ncol(sg),
                           reinterpret_cast<const float*>(params + h.off.b_o[sg]), C,
                           reinterpret_cast<float*>(bf.phi) + (int64_t)i0[sg] * C * Wo, Wo, (int64_t)N * C * Wo,
                           false};
      DQ_LAUNCH(h, kb + PK_GEMM_ORBITAL, gemm_tf32x3_tc_jobs(jd, 2, h.d_status, s));
    }
    for (int sg = 0; sg < 2 && !use_t3; ++sg) {
      if (ns[sg] == 0) continue;
      const RowMap mx{(int64_t)ns[sg] * C, (int64_t)N * C * D, D};
      const RowMap my{(int64_t)ns[sg] * C, (int64_t)N * C * Wo, Wo};
      {
        DQ_LAUNCH(h, kb + PK_GEMM_ORBITAL,
                  gemm_nt<T>(bf.F + (int64_t)i0[sg] * C * D, mx, params + h.off.W_o[sg], params + h.off.b_o[sg], C,
                             bf.phi + (int64_t)i0[sg] * C * Wo, my, nb * ns[sg] * C, K * h.ncol(sg), D, false, s));
      }
    }
    DQ_LAUNCH(h, kb + PK_ORBITAL_DET, launch_orbital_det<T>(h, d, params, bf, s));
    if (h.use_jastrow) {
      DQ_LAUNCH(h, kb + PK_JASTROW_SUM, launch_jastrow_sum<T>(h, d, bf, s));
      if (use_t3) {
        DQ_LAUNCH(h, kb + PK_GEMM_JASTROW,
                  gemm_tf32x3_tc_seg(reinterpret_cast<const float*>(bf.js), nb * C, 1, 0, D, D, w3.wj(0), w3.wj(1), D,
                                     reinterpret_cast<const float*>(params + h.off.b_J1), C,
                                     reinterpret_cast<float*>(bf.jh), D, 0, h.d_status, s));
      } else {
        const RowMap mj{(int64_t)C, (int64_t)C * D, D};
        DQ_LAUNCH(h, kb + PK_GEMM_JASTROW, gemm_nt<T>(bf.js, mj, params + h.off.W_J1, params + h.off.b_J1, C, bf.jh,
                                                      mj, nb * C, D, D, false, s));
      }
    }
    DQ_LAUNCH(h, kb + PK_COMBINE, launch_combine<T>(h, d, params, bf, logabs + b0, sign + b0,
                                                    e_loc ? e_loc + b0 : nullptr, s,
                                                    grad ? grad + b0 * 3 * N : nullptr));
  }
  return DQ_OK;
}

// ---------------------------------------------------------------------------
// grad_logpsi: value-only forward keeping every layer's activations, then the
// reverse pass (backward.cu).  Layout of the saved and adjoint buffers for a
// chunk of Bc walkers (C = 1, one row per node / edge / walker).
// ---------------------------------------------------------------------------
struct GradPlan {
  size_t geo, rbf, eh, ew, zl, msg, u, F, phi, det, js, jh, z0;  // saved forward
  size_t fbar, ubar, mbar, zbar, wbar, hbar, phibar, beta, cbar, jhbar, gt, sbar, envbar, ybar, part, done, wt3, wt3t;
  size_t ebar, abar;  // edge-embedding adjoints (iterated edge embeddings only)
  size_t h0, x0;      // hidden layer and inputs of the electron-nucleus initial embedding
  int64_t part_elems;
  size_t total;
};

GradPlan plan_grad(const dq_handle_s& h, int64_t Bc, size_t elem) {
  const int64_t E = h.edges.n_all, N = h.N, D = h.D, K = h.K, L = h.L, M = h.M, Q = h.Q;
  const int64_t nmax = h.det_n(), Wo = K * nmax;
  GradPlan p{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += align_up(bytes);
    return at;
  };
  p.geo = take(Bc * E * 4 * elem);
  p.rbf = take((h.edge_update ? L : 1) * Bc * E * Q * elem);  // every layer's edge embeddings when iterated
  p.eh = take(L * Bc * E * D * elem);
  p.ew = take(L * Bc * E * D * elem);
  p.zl = take(L * Bc * N * D * elem);
  p.msg = take(L * Bc * N * 3 * D * elem);
  p.u = take(L * Bc * N * D * elem);
  p.F = take((L + 1) * Bc * N * D * elem);
  p.phi = take(Bc * N * Wo * elem);
  p.det = take(Bc * 2 * K * (3 * N + 3) * sizeof(double));
  p.js = take(Bc * D * elem);
  p.jh = take(Bc * D * elem);
  p.z0 = take(2 * D * elem);
  p.fbar = take(Bc * N * D * elem);
  p.ubar = take(Bc * N * D * elem);
  p.mbar = take(Bc * N * 3 * D * elem);
  p.zbar = take(Bc * N * D * elem);
  p.wbar = take(Bc * E * D * elem);
  p.hbar = take(Bc * E * D * elem);
  p.phibar = take(Bc * N * Wo * elem);
  p.beta = take(Bc * K * elem);
  p.cbar = take(Bc * K * elem);
  p.jhbar = take(Bc * D * elem);
  p.gt = take(Bc * D * elem);
  p.sbar = take(Bc * D * elem);
  p.envbar = take(Bc * 2 * 2 * Wo * M * elem);
  p.ybar = take(Bc * M * D * elem);
  p.ebar = take(h.edge_update ? Bc * E * Q * elem : 0);
  p.h0 = take(h.el_init ? Bc * N * D * elem : 0);
  p.x0 = take(h.el_init ? Bc * N * 3 * M * elem : 0);
  p.abar = take(h.edge_update ? Bc * E * Q * elem : 0);
  const int64_t blk = std::max({3 * D * D, D * D, D * Q, Wo * D, Wo * M, M * D, K, D, Q * Q, 3 * M * D});
  p.part_elems = 64 * blk;
  p.part = take(p.part_elems * elem);
  p.done = take(kColsumReduceCounters * sizeof(unsigned int));
  p.wt3 = take(use_tf32x3(h) ? t3_weight_floats(h) * 4 : 0);
  p.wt3t = take(use_tf32x3(h) ? t3_weight_floats(h) * 4 : 0);  // transposed splits (reverse pass)
  p.total = o;
  return p;
}

inline RowMap rm(int64_t ld) { return RowMap{1, ld, 0}; }

template <class T>
dq_status run_grad(const dq_handle_s& h, const T* params, const T* r, int64_t B, const T* weights, int mode, T* G,
                   unsigned char* ws, size_t ws_bytes, cudaStream_t s) {
  const int64_t Bmax = std::min<int64_t>(B, h.max_chunk);
  const GradPlan pl = plan_grad(h, Bmax, sizeof(T));
  if (ws == nullptr || ws_bytes < pl.total || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  auto buf = [&](size_t off) { return reinterpret_cast<T*>(ws + off); };
  const int N = h.N, D = h.D, K = h.K, L = h.L, M = h.M, Q = h.Q, E = h.edges.n_all;
  const int Wo = K * h.det_n();
  const int64_t P = h.off.total;
  const ParamOffsets& off = h.off;
  const size_t el = sizeof(T);
  DQ_CU(cudaMemsetAsync(G, 0, (size_t)(mode == 1 ? B : 1) * P * el, s));
  T* part = buf(pl.part);
  unsigned int* done = reinterpret_cast<unsigned int*>(ws + pl.done);
  DQ_CU(cudaMemsetAsync(done, 0, kColsumReduceCounters * sizeof(unsigned int), s));
  const bool use_t3 = sizeof(T) == 4 && use_tf32x3(h);
  const T3Weights w3 = t3_weights(h, ws + pl.wt3);
  // transposed splits for the products with W in the reverse pass (same block layout per layer)
  const T3Weights w3t = t3_weights(h, ws + pl.wt3t);
  if (use_t3) {
    if constexpr (sizeof(T) == 4) {
      DQ_CU(split_t3_weights(h, params, w3, s));
      for (int l = 0; l < L; ++l) {
        const auto& y = off.layer[l];
        DQ_CU(split_tf32_t(params + y.W_g, D, 3 * D, w3t.wg(l, 0), w3t.wg(l, 1), s));
        DQ_CU(split_tf32_t(params + y.W_h, D, D, w3t.wh(l, 0), w3t.wh(l, 1), s));
        for (int t = 0; t < 3; ++t) DQ_CU(split_tf32_t(params + y.W2[t], D, D, w3t.w2(l, t, 0), w3t.w2(l, t, 1), s));
      }
      const int nsp[2] = {h.n_up, h.n_dn};
      for (int sg = 0; sg < 2; ++sg)
        if (nsp[sg] > 0) DQ_CU(split_tf32_t(params + off.W_o[sg], K * h.ncol(sg), D, w3t.wo(sg, 0), w3t.wo(sg, 1), s));
    }
  }
  const int ns[2] = {h.n_up, h.n_dn}, i0[2] = {0, h.n_up};
  const int e0[3] = {0, h.edges.n_par, h.edges.n_ee};
  const int ng[3] = {h.edges.n_par, h.edges.n_anti, h.edges.n_en};
  for (int64_t b0 = 0; b0 < B; b0 += Bmax) {
    const int64_t nb = std::min<int64_t>(Bmax, B - b0);
    const FwdDims d{nb, N, h.n_up, h.n_dn, M, D, K, Q, 1};
    T* Gc = mode == 1 ? G + b0 * P : G;
    const T* wc = weights ? weights + b0 : nullptr;
    auto reduce = [&](const T* X, RowMap mx, const T* Y, RowMap my, int rpw, int n_o, int n_a, int64_t poff, int ld) {
      return param_reduce<T>(X, mx, Y, my, rpw, nb, n_o, n_a, Gc, P, poff, ld, mode, part, pl.part_elems, s,
                             use_t3 ? h.d_status : nullptr, done);
    };
    // a weight gradient X^T Y and the bias gradient sum_r X[r] of the same adjoint X: one pass over X
    // where the tensor-core reduction runs, else a column-sum launch for the bias
    auto reduce_wb = [&](const T* X, RowMap mx, const T* Y, RowMap my, int rpw, int n_o, int n_a, int64_t woff,
                         int ld, int64_t boff) {
      bool bias_done = false;
      cudaError_t e = param_reduce<T>(X, mx, Y, my, rpw, nb, n_o, n_a, Gc, P, woff, ld, mode, part, pl.part_elems, s,
                                      use_t3 ? h.d_status : nullptr, done, boff, &bias_done);
      if (e == cudaSuccess && !bias_done) e = reduce(X, mx, nullptr, rm(1), rpw, n_o, 1, boff, 1);
      return e;
    };
    // ---- forward, keeping activations ----
    FwdBuffers<T> v{};
    v.geo = buf(pl.geo);
    v.rbf = buf(pl.rbf);
    v.phi = buf(pl.phi);
    v.det = reinterpret_cast<double*>(ws + pl.det);
    v.js = buf(pl.js);
    v.jh = buf(pl.jh);
    v.z0 = buf(pl.z0);
    auto EH = [&](int l) { return buf(pl.eh) + (int64_t)l * Bmax * E * D; };
    auto EW = [&](int l) { return buf(pl.ew) + (int64_t)l * Bmax * E * D; };
    auto ZL = [&](int l) { return buf(pl.zl) + (int64_t)l * Bmax * N * D; };
    auto MS = [&](int l) { return buf(pl.msg) + (int64_t)l * Bmax * N * 3 * D; };
    auto U = [&](int l) { return buf(pl.u) + (int64_t)l * Bmax * N * D; };
    auto F = [&](int l) { return buf(pl.F) + (int64_t)l * Bmax * N * D; };
    // edge embeddings of layer l (one shared buffer unless they are iterated)
    auto RB = [&](int l) { return buf(pl.rbf) + (h.edge_update ? (int64_t)l * Bmax * E * Q : 0); };
    if (!h.el_init) DQ_LAUNCH(h, kValueOffset + PK_LAYER0, launch_layer0_node<T>(h, d, params, v, s));
    DQ_LAUNCH(h, kValueOffset + PK_GEOMETRY, launch_geometry<T>(h, d, r + b0 * N * 3, v, s));
    if (h.el_init)
      DQ_LAUNCH(h, kValueOffset + PK_LAYER0, launch_el_init<T>(h, d, params, r + b0 * N * 3, F(0), nullptr,
                                                              buf(pl.h0), buf(pl.x0), s));
    else
      DQ_LAUNCH(h, kValueOffset + PK_UPDATE, launch_fill_spin_rows<T>(F(0), params + off.E_spin, nb, N, h.n_up, D, s));
    const bool spin0 = !h.el_init;  // layer 0 on the spin embeddings (constant z, f^0 from E_spin)
    for (int l = 0; l < L; ++l) {
      const auto& y = off.layer[l];
      v.eh = EH(l);
      v.ew = EW(l);
      v.F = F(l);
      v.Z = ZL(l);
      v.msg = MS(l);
      if (h.edge_update && l > 0)
        DQ_LAUNCH(h, kValueOffset + PK_EDGE_HIDDEN, launch_edge_update<T>(h, d, params, l, RB(l - 1), RB(l), s));
      v.rbf = RB(l);
      DQ_LAUNCH(h, kValueOffset + PK_EDGE_HIDDEN, launch_edge_hidden<T>(h, d, params, l, v, s));
      for (int t = 0; t < 3; ++t) {
        if (ng[t] == 0) continue;
        const RowMap m{(int64_t)ng[t], (int64_t)E * D, D};
        if (use_t3) {
          DQ_LAUNCH(h, kValueOffset + PK_GEMM_EDGE,
                    gemm_tf32x3_tc_seg(reinterpret_cast<const float*>(v.eh) + (int64_t)e0[t] * D, ng[t], nb,
                                       (int64_t)E * D, D, D, w3.w2(l, t, 0), w3.w2(l, t, 1), D,
                                       reinterpret_cast<const float*>(params + y.b2[t]), 1,
                                       reinterpret_cast<float*>(v.ew) + (int64_t)e0[t] * D, D, (int64_t)E * D,
                                       h.d_status, s));
        } else {
          DQ_LAUNCH(h, kValueOffset + PK_GEMM_EDGE,
                    gemm_nt<T>(v.eh + (int64_t)e0[t] * D, m, params + y.W2[t], params + y.b2[t], 1,
                               v.ew + (int64_t)e0[t] * D, m, nb * ng[t], D, D, false, s));
        }
      }
      if ((l > 0 || !spin0) && use_t3)
        DQ_LAUNCH(h, kValueOffset + PK_GEMM_NODE,
                  gemm_tf32x3_tc(reinterpret_cast<const float*>(F(l)), nb * N, D, D, w3.wh(l, 0), w3.wh(l, 1), D,
                                 nullptr, 1, reinterpret_cast<float*>(ZL(l)), D, h.d_status, s));
      else if (l > 0 || !spin0)
        DQ_LAUNCH(h, kValueOffset + PK_GEMM_NODE, gemm_nt<T>(F(l), rm(D), params + y.W_h, nullptr, 1, ZL(l), rm(D), nb * N, D, D,
                                             false, s));
      DQ_LAUNCH(h, kValueOffset + PK_MESSAGES, launch_messages<T>(h, d, params, l, l == 0 && spin0, v, s));
      if (use_t3)
        DQ_LAUNCH(h, kValueOffset + PK_GEMM_UPDATE,
                  gemm_tf32x3_tc(reinterpret_cast<const float*>(MS(l)), nb * N, 3 * D, 3 * D, w3.wg(l, 0),
                                 w3.wg(l, 1), D, reinterpret_cast<const float*>(params + y.b_g), 1,
                                 reinterpret_cast<float*>(U(l)), D, h.d_status, s));
      else
        DQ_LAUNCH(h, kValueOffset + PK_GEMM_UPDATE, gemm_nt<T>(MS(l), rm(3 * D), params + y.W_g, params + y.b_g, 1, U(l), rm(D), nb * N,
                                           D, 3 * D, false, s));
      DQ_LAUNCH(h, kValueOffset + PK_UPDATE, launch_update_io<T>(h, d, params, l == 0 && spin0, U(l), F(l), F(l + 1), s));
    }
    v.F = F(L);
    for (int sg = 0; sg < 2; ++sg) {
      if (ns[sg] == 0) continue;
      const RowMap mx{(int64_t)ns[sg], (int64_t)N * D, D};
      const RowMap my{(int64_t)ns[sg], (int64_t)N * Wo, Wo};
      if (use_t3)
        DQ_LAUNCH(h, kValueOffset + PK_GEMM_ORBITAL,
                  gemm_tf32x3_tc_seg(reinterpret_cast<const float*>(F(L)) + (int64_t)i0[sg] * D, ns[sg], nb,
                                     (int64_t)N * D, D, D, w3.wo(sg, 0), w3.wo(sg, 1), K * h.ncol(sg),
                                     reinterpret_cast<const float*>(params + off.b_o[sg]), 1,
                                     reinterpret_cast<float*>(v.phi) + (int64_t)i0[sg] * Wo, Wo, (int64_t)N * Wo,
                                     h.d_status, s));
      else
        DQ_LAUNCH(h, kValueOffset + PK_GEMM_ORBITAL, gemm_nt<T>(F(L) + (int64_t)i0[sg] * D, mx, params + off.W_o[sg], params + off.b_o[sg],
                                           1, v.phi + (int64_t)i0[sg] * Wo, my, nb * ns[sg], K * h.ncol(sg), D, false, s));
    }
    DQ_LAUNCH(h, kValueOffset + PK_ORBITAL_DET, launch_orbital_det<T>(h, d, params, v, s));
    if (h.use_jastrow) {
      DQ_LAUNCH(h, kValueOffset + PK_JASTROW_SUM, launch_jastrow_sum<T>(h, d, v, s));
      DQ_LAUNCH(h, kValueOffset + PK_GEMM_JASTROW, gemm_nt<T>(v.js, rm(D), params + off.W_J1, params + off.b_J1, 1, v.jh, rm(D), nb, D, D,
                                           false, s));
    }
    // ---- reverse pass ----
    T *beta = buf(pl.beta), *cbar = buf(pl.cbar), *jhbar = buf(pl.jhbar), *gt = buf(pl.gt), *sbar = buf(pl.sbar);
    T *fbar = buf(pl.fbar), *ubar = buf(pl.ubar), *mbar = buf(pl.mbar), *zbar = buf(pl.zbar);
    T *wbar = buf(pl.wbar), *hbar = buf(pl.hbar), *phibar = buf(pl.phibar), *envbar = buf(pl.envbar);
    T* ybar = buf(pl.ybar);
    T* ebar = h.edge_update ? buf(pl.ebar) : nullptr;
    T* abar = h.edge_update ? buf(pl.abar) : nullptr;
    if (h.edge_update) DQ_CU(cudaMemsetAsync(ebar, 0, (size_t)nb * E * Q * sizeof(T), s));
    DQ_LAUNCH(h, PK_BWD_COMBINE,
              launch_bwd_combine<T>(h, nb, v.det, v.jh, params, wc, beta, cbar, jhbar, gt, s));
    DQ_LAUNCH(h, PK_BWD_REDUCE, reduce(cbar, rm(K), nullptr, rm(1), 1, K, 1, off.c, 1));
    if (h.use_jastrow) {
      DQ_LAUNCH(h, PK_BWD_REDUCE, reduce(gt, rm(D), nullptr, rm(1), 1, D, 1, off.w_J2, 1));
      DQ_LAUNCH(h, PK_BWD_REDUCE, reduce(jhbar, rm(D), v.js, rm(D), 1, D, D, off.W_J1, D));
      DQ_LAUNCH(h, PK_BWD_REDUCE, reduce(jhbar, rm(D), nullptr, rm(1), 1, D, 1, off.b_J1, 1));
      DQ_LAUNCH(h, PK_BWD_GEMM, gemm_nn<T>(jhbar, rm(D), params + off.W_J1, sbar, rm(D), nb, D, D, false, s));
    }
    DQ_LAUNCH(h, PK_BWD_DET, launch_bwd_det<T>(h, nb, v.phi, v.geo, params, beta, phibar, envbar, s));
    for (int sg = 0; sg < 2; ++sg) {
      if (ns[sg] == 0) continue;
      const int64_t blk = (int64_t)Wo * M;
      const RowMap me{1, 4 * blk, 0};
      const int nc = K * h.ncol(sg);  // orbitals of this spin's network
      DQ_LAUNCH(h, PK_BWD_REDUCE, reduce(envbar + (sg * 2 + 0) * blk, me, nullptr, rm(1), 1, nc * M, 1,
                                         off.omega[sg], 1));
      DQ_LAUNCH(h, PK_BWD_REDUCE, reduce(envbar + (sg * 2 + 1) * blk, me, nullptr, rm(1), 1, nc * M, 1,
                                         off.zeta[sg], 1));
      const RowMap mp{(int64_t)ns[sg], (int64_t)N * Wo, Wo};
      const RowMap mf{(int64_t)ns[sg], (int64_t)N * D, D};
      const T* pb = phibar + (int64_t)i0[sg] * Wo;
      DQ_LAUNCH(h, PK_BWD_REDUCE, reduce_wb(pb, mp, F(L) + (int64_t)i0[sg] * D, mf, ns[sg], nc, D, off.W_o[sg], D,
                                            off.b_o[sg]));
      // tensor cores when the rows of phi-bar suit the tensor maps (K * n_c and Wo multiples of 4)
      if (use_t3 && nc % 4 == 0 && Wo % 4 == 0)
        DQ_LAUNCH(h, PK_BWD_GEMM,
                  gemm_tf32x3_tc_seg(reinterpret_cast<const float*>(pb), ns[sg], nb, (int64_t)N * Wo, nc, Wo,
                                     w3t.wo(sg, 0), w3t.wo(sg, 1), D, nullptr, 1,
                                     reinterpret_cast<float*>(fbar) + (int64_t)i0[sg] * D, D, (int64_t)N * D,
                                     h.d_status, s));
      else
        DQ_LAUNCH(h, PK_BWD_GEMM, gemm_nn<T>(pb, mp, params + off.W_o[sg], fbar + (int64_t)i0[sg] * D, mf,
                                           nb * ns[sg], D, nc, false, s));
    }
    if (h.use_jastrow) DQ_LAUNCH(h, PK_BWD_UPDATE, launch_add_rows<T>(fbar, sbar, nb, N, D, s));
    for (int l = L - 1; l >= 0; --l) {
      const auto& y = off.layer[l];
      DQ_LAUNCH(h, PK_BWD_UPDATE, launch_tanh_bwd<T>(fbar, U(l), nb * N * D, true, ubar, s));
      DQ_LAUNCH(h, PK_BWD_REDUCE, reduce_wb(ubar, rm(D), MS(l), rm(3 * D), N, D, 3 * D, y.W_g, 3 * D, y.b_g));
      if (use_t3)
        DQ_LAUNCH(h, PK_BWD_GEMM,
                  gemm_tf32x3_tc(reinterpret_cast<const float*>(ubar), nb * N, D, D, w3t.wg(l, 0), w3t.wg(l, 1),
                                 3 * D, nullptr, 1, reinterpret_cast<float*>(mbar), 3 * D, h.d_status, s));
      else
        DQ_LAUNCH(h, PK_BWD_GEMM, gemm_nn<T>(ubar, rm(D), params + y.W_g, mbar, rm(3 * D), nb * N, 3 * D, D, false, s));
      DQ_LAUNCH(h, PK_BWD_MESSAGES, launch_msg_bwd<T>(h, nb, mbar, ZL(l), v.z0, EW(l), params + y.Y, l == 0 && spin0,
                                                      zbar, wbar, ybar, s));
      DQ_LAUNCH(h, PK_BWD_REDUCE, reduce(ybar, rm((int64_t)M * D), nullptr, rm(1), 1, M * D, 1, y.Y, 1));
      DQ_LAUNCH(h, PK_BWD_REDUCE, reduce(zbar, rm(D), F(l), rm(D), N, D, D, y.W_h, D));
      if (use_t3)
        DQ_LAUNCH(h, PK_BWD_GEMM,
                  gemm_tf32x3_tc_seg(reinterpret_cast<const float*>(zbar), nb * N, 1, 0, D, D, w3t.wh(l, 0),
                                     w3t.wh(l, 1), D, nullptr, 1, reinterpret_cast<float*>(fbar), D, 0, h.d_status, s,
                                     true));
      else
        DQ_LAUNCH(h, PK_BWD_GEMM, gemm_nn<T>(zbar, rm(D), params + y.W_h, fbar, rm(D), nb * N, D, D, true, s));
      for (int t = 0; t < 3; ++t) {
        if (ng[t] == 0) continue;
        const RowMap me{(int64_t)ng[t], (int64_t)E * D, D};
        const T* wb = wbar + (int64_t)e0[t] * D;
        DQ_LAUNCH(h, PK_BWD_REDUCE, reduce_wb(wb, me, EH(l) + (int64_t)e0[t] * D, me, ng[t], D, D, y.W2[t], D,
                                              y.b2[t]));
        if (use_t3)
          DQ_LAUNCH(h, PK_BWD_GEMM,
                    gemm_tf32x3_tc_seg(reinterpret_cast<const float*>(wb), ng[t], nb, (int64_t)E * D, D, D,
                                       w3t.w2(l, t, 0), w3t.w2(l, t, 1), D, nullptr, 1,
                                       reinterpret_cast<float*>(hbar) + (int64_t)e0[t] * D, D, (int64_t)E * D,
                                       h.d_status, s));
        else
          DQ_LAUNCH(h, PK_BWD_GEMM, gemm_nn<T>(wb, me, params + y.W2[t], hbar + (int64_t)e0[t] * D, me, nb * ng[t], D, D,
                                             false, s));
      }
      DQ_LAUNCH(h, PK_BWD_EDGE, launch_tanh_bwd<T>(hbar, EH(l), nb * E * D, false, hbar, s));
      for (int t = 0; t < 3; ++t) {
        if (ng[t] == 0) continue;
        const RowMap me{(int64_t)ng[t], (int64_t)E * D, D};
        const RowMap mq{(int64_t)ng[t], (int64_t)E * Q, Q};
        const T* hb = hbar + (int64_t)e0[t] * D;
        DQ_LAUNCH(h, PK_BWD_REDUCE, reduce_wb(hb, me, RB(l) + (int64_t)e0[t] * Q, mq, ng[t], D, Q, y.W1[t], Q,
                                              y.b1[t]));
        if (h.edge_update && l > 0)  // adjoint of this layer's edge embeddings: W1^T h-bar
          DQ_LAUNCH(h, PK_BWD_GEMM, gemm_nn<T>(hb, me, params + y.W1[t], ebar + (int64_t)e0[t] * Q, mq,
                                             nb * ng[t], Q, D, true, s));
      }
      if (h.edge_update && l > 0) {  // through f^l = f^{l-1} + tanh(U f^{l-1} + c) (Eq. 16)
        DQ_LAUNCH(h, PK_BWD_EDGE, launch_edge_update_bwd<T>(h, nb, l, params, RB(l - 1), ebar, abar, s));
        for (int t = 0; t < 3; ++t) {
          if (ng[t] == 0) continue;
          const RowMap mq{(int64_t)ng[t], (int64_t)E * Q, Q};
          const T* ab = abar + (int64_t)e0[t] * Q;
          DQ_LAUNCH(h, PK_BWD_REDUCE, reduce_wb(ab, mq, RB(l - 1) + (int64_t)e0[t] * Q, mq, ng[t], Q, Q, y.U[t], Q,
                                                y.c[t]));
        }
      }
    }
    if (h.el_init) {  // through f^0 = W_e2 tanh(W_e1 x + b_e1) + b_e2 (Eq. 13, second case)
      const int M3 = 3 * M;
      T* H0 = buf(pl.h0);
      DQ_LAUNCH(h, PK_BWD_REDUCE, reduce_wb(fbar, rm(D), H0, rm(D), N, D, D, off.W_e2, D, off.b_e2));
      DQ_LAUNCH(h, PK_BWD_GEMM, gemm_nn<T>(fbar, rm(D), params + off.W_e2, ubar, rm(D), nb * N, D, D, false, s));
      DQ_LAUNCH(h, PK_BWD_UPDATE, launch_tanh_bwd<T>(ubar, H0, nb * N * D, false, ubar, s));
      DQ_LAUNCH(h, PK_BWD_REDUCE, reduce_wb(ubar, rm(D), buf(pl.x0), rm(M3), N, D, M3, off.W_e1, M3, off.b_e1));
    } else {
      for (int sg = 0; sg < 2; ++sg) {
        if (ns[sg] == 0) continue;
        const RowMap mf{(int64_t)ns[sg], (int64_t)N * D, D};
        DQ_LAUNCH(h, PK_BWD_REDUCE, reduce(fbar + (int64_t)i0[sg] * D, mf, nullptr, rm(1), ns[sg], D, 1,
                                           off.E_spin + (int64_t)sg * D, 1));
      }
    }
  }
  return DQ_OK;
}

dq_status check_handle(dq_handle h) {
  if (h == nullptr) return DQ_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return DQ_ERR_CUDA;
  if (dev != h->device) return DQ_ERR_ARG;
  return DQ_OK;
}

}  // namespace
}  // namespace dq

namespace dq {
namespace {
template <class T>
dq_status run_mcmc(dq_handle h, const T* params, T* r, T* logabs, int64_t B, int32_t n_steps, double step,
                   uint64_t seed, uint64_t t0, uint64_t* t_dev, int64_t* n_acc, unsigned char* ws, size_t ws_bytes,
                   cudaStream_t s) {
  const McmcPlan plan = plan_mcmc(*h, B, sizeof(T));
  if (ws == nullptr || ws_bytes < plan.total || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  T* r_prop = reinterpret_cast<T*>(ws + plan.r_prop);
  T* la_prop = reinterpret_cast<T*>(ws + plan.la_prop);
  int8_t* sg_prop = reinterpret_cast<int8_t*>(ws + plan.sign_prop);
  if (n_acc) DQ_CU(cudaMemsetAsync(n_acc, 0, sizeof(int64_t), s));
  for (int32_t k = 0; k < n_steps; ++k) {
    const uint64_t t = t0 + (uint64_t)k;
    DQ_LAUNCH(*h, PK_PROPOSE, launch_propose<T>(*h, B, r, r_prop, step, seed, t, t_dev, s));
    dq_status st = run_forward<T>(*h, params, r_prop, B, false, la_prop, sg_prop, nullptr, ws + plan.fwd,
                                  ws_bytes - plan.fwd, s);
    if (st != DQ_OK) return st;
    DQ_LAUNCH(*h, PK_ACCEPT, launch_accept<T>(*h, B, r, logabs, r_prop, la_prop, sg_prop, seed, t, t_dev,
                           reinterpret_cast<unsigned long long*>(n_acc), s));
  }
  if (t_dev) DQ_CU(launch_advance_counter(t_dev, (uint64_t)n_steps, s));
  return DQ_OK;
}

// Metropolis steps whose proposals are evaluated by the jets forward: the same proposals, uniforms
// and acceptance as run_mcmc, with the proposal's local energy carried to accepted walkers.
template <class T>
dq_status run_mcmc_eloc(dq_handle h, const T* params, T* r, T* logabs, T* e_loc, int64_t B, int32_t n_steps,
                        double step, uint64_t seed, uint64_t t0, uint64_t* t_dev, int64_t* n_acc, unsigned char* ws,
                        size_t ws_bytes, cudaStream_t s) {
  const MalaPlan plan = plan_mala(*h, B, sizeof(T));
  if (ws == nullptr || ws_bytes < plan.total || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  T* r_prop = reinterpret_cast<T*>(ws + plan.r_prop);
  T* la_prop = reinterpret_cast<T*>(ws + plan.la_prop);
  int8_t* sg_prop = reinterpret_cast<int8_t*>(ws + plan.sign_prop);
  T* e_prop = reinterpret_cast<T*>(ws + plan.e_prop);
  if (n_acc) DQ_CU(cudaMemsetAsync(n_acc, 0, sizeof(int64_t), s));
  for (int32_t k = 0; k < n_steps; ++k) {
    const uint64_t t = t0 + (uint64_t)k;
    DQ_LAUNCH(*h, PK_PROPOSE, launch_propose<T>(*h, B, r, r_prop, step, seed, t, t_dev, s));
    dq_status st = run_forward<T>(*h, params, r_prop, B, true, la_prop, sg_prop, e_prop, ws + plan.fwd,
                                  ws_bytes - plan.fwd, s);
    if (st != DQ_OK) return st;
    DQ_LAUNCH(*h, PK_ACCEPT, launch_accept<T>(*h, B, r, logabs, r_prop, la_prop, sg_prop, seed, t, t_dev,
                                              reinterpret_cast<unsigned long long*>(n_acc), s, e_loc, e_prop));
  }
  if (t_dev && n_steps > 0) DQ_CU(launch_advance_counter(t_dev, (uint64_t)n_steps, s));
  return DQ_OK;
}

template <class T>
dq_status run_mala(dq_handle h, const T* params, T* r, T* logabs, T* grad, T* e_loc, int grad_valid, int64_t B,
                   int32_t n_steps, double tau, uint64_t seed, uint64_t t0, uint64_t* t_dev, int64_t* n_acc,
                   unsigned char* ws, size_t ws_bytes, cudaStream_t s) {
  const MalaPlan plan = plan_mala(*h, B, sizeof(T));
  if (ws == nullptr || ws_bytes < plan.total || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  T* r_prop = reinterpret_cast<T*>(ws + plan.r_prop);
  T* la_prop = reinterpret_cast<T*>(ws + plan.la_prop);
  int8_t* sg_prop = reinterpret_cast<int8_t*>(ws + plan.sign_prop);
  T* g_prop = reinterpret_cast<T*>(ws + plan.g_prop);
  T* xi = reinterpret_cast<T*>(ws + plan.xi);
  T* e_prop = reinterpret_cast<T*>(ws + plan.e_prop);
  if (n_acc) DQ_CU(cudaMemsetAsync(n_acc, 0, sizeof(int64_t), s));
  if (!grad_valid) {  // d log|psi| / d r at the starting positions (log|psi| recomputed too)
    dq_status st = run_forward<T>(*h, params, r, B, true, logabs, sg_prop, e_loc ? e_loc : e_prop, ws + plan.fwd,
                                  ws_bytes - plan.fwd, s, grad);
    if (st != DQ_OK) return st;
  }
  for (int32_t k = 0; k < n_steps; ++k) {
    const uint64_t t = t0 + (uint64_t)k;
    DQ_LAUNCH(*h, PK_PROPOSE, launch_mala_propose<T>(*h, B, r, grad, r_prop, xi, tau, seed, t, t_dev, s));
    dq_status st = run_forward<T>(*h, params, r_prop, B, true, la_prop, sg_prop, e_prop, ws + plan.fwd,
                                  ws_bytes - plan.fwd, s, g_prop);
    if (st != DQ_OK) return st;
    DQ_LAUNCH(*h, PK_ACCEPT, launch_mala_accept<T>(*h, B, r, logabs, grad, r_prop, la_prop, sg_prop, g_prop, xi, e_loc,
                                                   e_prop, tau, seed, t, t_dev,
                                                   reinterpret_cast<unsigned long long*>(n_acc), s));
  }
  if (t_dev && n_steps > 0) DQ_CU(launch_advance_counter(t_dev, (uint64_t)n_steps, s));
  return DQ_OK;
}
// ---------------------------------------------------------------------------
// Batches of molecules (dq_multi): every kernel of the forward pass, the
// sampler and the loss weights runs as one launch over all molecules of the
// batch (grouped launches, forward.cu / mcmc.cu; the 3 x TF32 GEMMs as one
// persistent job-list launch), each molecule with its own electron count,
// parameters and buffers.  Walkers are processed in `rounds` chunks: molecule m
// takes ceil(B_m / rounds) walkers per round.
// ---------------------------------------------------------------------------
struct MultiFwdPlan {
  int rounds;
  int64_t Bc[kMaxGroup];
  size_t off[kMaxGroup];
  FwdPlan fp[kMaxGroup];
  size_t total;
};

int multi_rounds(const dq_multi_s& g, const int64_t* B) {
  if (g.rounds > 0) return g.rounds;
  int r = 1;
  for (int m = 0; m < g.n; ++m) r = std::max<int>(r, (int)((B[m] + g.h[m]->max_chunk - 1) / g.h[m]->max_chunk));
  return r;
}

MultiFwdPlan plan_forward_multi(const dq_multi_s& g, const int64_t* B, bool jets, size_t elem) {
  MultiFwdPlan p{};
  p.rounds = multi_rounds(g, B);
  size_t o = 0;
  for (int m = 0; m < g.n; ++m) {
    p.Bc[m] = std::max<int64_t>(1, (std::max<int64_t>(B[m], 0) + p.rounds - 1) / p.rounds);
    p.fp[m] = plan_forward(*g.h[m], p.Bc[m], jets, elem);
    p.off[m] = o;
    o += align_up(p.fp[m].total);
  }
  p.total = o;
  return p;
}

template <class T>
FwdBuffers<T> carve_forward(const FwdPlan& plan, unsigned char* ws, bool bf16) {
  FwdBuffers<T> bf;
  bf.geo = reinterpret_cast<T*>(ws + plan.geo);
  bf.rbf = reinterpret_cast<T*>(ws + plan.rbf);
  bf.eh = reinterpret_cast<T*>(ws + plan.eh);
  bf.ew = reinterpret_cast<T*>(ws + plan.ew);
  bf.F = reinterpret_cast<T*>(ws + plan.F);
  bf.Z = reinterpret_cast<T*>(ws + plan.Z);
  bf.msg = reinterpret_cast<T*>(ws + plan.msg);
  bf.phi = reinterpret_cast<T*>(ws + plan.phi);
  bf.det = reinterpret_cast<double*>(ws + plan.det);
  bf.js = reinterpret_cast<T*>(ws + plan.js);
  bf.jh = reinterpret_cast<T*>(ws + plan.jh);
  bf.z0 = reinterpret_cast<T*>(ws + plan.z0);
  bf.msg_bf = bf16 ? ws + plan.msg_bf : nullptr;
  bf.F_bf = bf16 ? ws + plan.F_bf : nullptr;
  return bf;
}

// The forward pass of a batch: per walker the same kernels and GEMM tiles as
// run_forward (which launches the same grouped kernels with one entry), so each
// molecule's results equal its single-molecule results bit for bit.
template <class T>
dq_status run_forward_multi(const dq_multi_s& g, const T* const* params, const T* const* r, const int64_t* B,
                            bool jets, T* const* logabs, int8_t* const* sign, T* const* e_loc, unsigned char* ws,
                            size_t ws_bytes, cudaStream_t s, const MultiFwdPlan* given = nullptr) {
  static_assert(sizeof(T) == 4, "batches run in the FP32 modes");
  const int n = g.n;
  const MultiFwdPlan P = given ? *given : plan_forward_multi(g, B, jets, sizeof(T));
  if (ws == nullptr || ws_bytes < P.total || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  const dq_handle_s& H = *g.h[0];  // launch timing of the batch goes to molecule 0's profiler
  const bool use_tc = g.precision == DQ_BF16_MIXED;
  MolFwd<T> mf[kMaxGroup];
  T3Weights w3[kMaxGroup];
  unsigned char* Wbf[kMaxGroup];
  for (int m = 0; m < n; ++m) {
    const dq_handle_s& h = *g.h[m];
    unsigned char* base = ws + P.off[m];
    mf[m].h = &h;
    mf[m].params = params[m];
    mf[m].b = carve_forward<T>(P.fp[m], base, use_tc);
    const int C = jets ? 3 * h.N + 2 : 1;
    mf[m].d = FwdDims{P.Bc[m], h.N, h.n_up, h.n_dn, h.M, h.D, h.K, h.Q, C};
    w3[m] = t3_weights(h, base + P.fp[m].W_t3);
    DQ_CU(split_t3_weights(h, params[m], w3[m], s));
    Wbf[m] = base + P.fp[m].W_bf;
    if (use_tc)
      for (int l = 0; l < h.L; ++l) {
        DQ_CU(launch_to_bf16(params[m] + h.off.layer[l].W_g, Wbf[m] + (size_t)l * 4 * h.D * h.D * 2,
                             (int64_t)3 * h.D * h.D, s));
        DQ_CU(launch_to_bf16(params[m] + h.off.layer[l].W_h, Wbf[m] + ((size_t)l * 4 + 3) * h.D * h.D * 2,
                             (int64_t)h.D * h.D, s));
      }
  }
  const int kb = jets ? 0 : kValueOffset;
  const int L = g.h[0]->L;
  DQ_LAUNCH(H, kb + PK_LAYER0, launch_layer0_node_group<T>(mf, n, s));
  const T* rq[kMaxGroup];
  T *la[kMaxGroup], *el[kMaxGroup];
  int8_t* sg[kMaxGroup];
  T3JobDesc jd[6 * kMaxGroup];
  for (int q = 0; q < P.rounds; ++q) {
    bool any = false;
    for (int m = 0; m < n; ++m) {
      const dq_handle_s& h = *g.h[m];
      const int64_t b0 = (int64_t)q * P.Bc[m];
      const int64_t nb = std::max<int64_t>(0, std::min<int64_t>(P.Bc[m], B[m] - b0));
      mf[m].d.Bc = nb;
      any = any || nb > 0;
      rq[m] = nb > 0 ? r[m] + b0 * h.N * 3 : nullptr;
      la[m] = nb > 0 ? logabs[m] + b0 : nullptr;
      sg[m] = nb > 0 ? sign[m] + b0 : nullptr;
      el[m] = nb > 0 && e_loc ? e_loc[m] + b0 : nullptr;
    }
    if (!any) break;
    DQ_LAUNCH(H, kb + PK_GEOMETRY, launch_geometry_group<T>(mf, n, rq, s));
    for (int m = 0; m < n; ++m)  // electron-nucleus initial embeddings (Eq. 13, second case)
      if (g.h[m]->el_init && mf[m].d.Bc > 0)
        DQ_LAUNCH(H, kb + PK_LAYER0, launch_el_init<T>(*g.h[m], mf[m].d, params[m], rq[m], mf[m].b.F,
                                                      use_tc ? mf[m].b.F_bf : nullptr, nullptr, nullptr, s));
    for (int l = 0; l < L; ++l) {
      if (l > 0) {  // iterated edge embeddings of the molecules that have them, in place
        const T* es[kMaxGroup];
        T* ed[kMaxGroup];
        bool anyu = false;
        for (int m = 0; m < n; ++m) {
          es[m] = ed[m] = mf[m].b.rbf;
          anyu = anyu || (g.h[m]->edge_update && mf[m].d.Bc > 0);
        }
        if (anyu) DQ_LAUNCH(H, kb + PK_EDGE_HIDDEN, launch_edge_update_group<T>(mf, n, l, es, ed, s));
      }
      DQ_LAUNCH(H, kb + PK_EDGE_HIDDEN, launch_edge_hidden_group<T>(mf, n, l, s));
      int nj = 0;
      for (int m = 0; m < n; ++m) {  // edge filters: three edge types of every molecule
        const dq_handle_s& h = *g.h[m];
        const FwdDims& d = mf[m].d;
        if (d.Bc <= 0) continue;
        const int ej = d.C > 1 ? 3 : 1, E = h.edges.n_all, D = h.D;
        const int e0[3] = {0, h.edges.n_par, h.edges.n_ee};
        const int ng[3] = {h.edges.n_par, h.edges.n_anti, h.edges.n_en};
        const int64_t seg = (int64_t)E * ej * D;
        for (int t = 0; t < 3; ++t)
          jd[nj++] = T3JobDesc{reinterpret_cast<const float*>(mf[m].b.eh) + (int64_t)e0[t] * ej * D,
                               (int64_t)ng[t] * ej, d.Bc, seg, D, D, w3[m].w2(l, t, 0), w3[m].w2(l, t, 1), D,
                               reinterpret_cast<const float*>(params[m] + h.off.layer[l].b2[t]), ej,
                               reinterpret_cast<float*>(mf[m].b.ew) + (int64_t)e0[t] * ej * D, D, seg, false};
      }
      DQ_LAUNCH(H, kb + PK_GEMM_EDGE, gemm_tf32x3_tc_jobs(jd, nj, H.d_status, s));
      {  // node map z = W_h f (layer 0 only for the molecules without spin embeddings)
        nj = 0;
        for (int m = 0; m < n; ++m) {
          const dq_handle_s& h = *g.h[m];
          const FwdDims& d = mf[m].d;
          if (d.Bc <= 0 || (l == 0 && !h.el_init)) continue;
          const int64_t rows = d.Bc * d.N * d.C;
          if (use_tc && !use_fused(h, jets)) {  // (fused molecules: 3 x TF32, as in their single calls)
            DQ_LAUNCH(H, kb + PK_GEMM_NODE,
                      gemm_bf16_tc(mf[m].b.F_bf, rows, h.D, h.D, Wbf[m] + ((size_t)l * 4 + 3) * h.D * h.D * 2, h.D,
                                   nullptr, 1, reinterpret_cast<float*>(mf[m].b.Z), h.D, H.d_status, s));
          } else {
            jd[nj++] = T3JobDesc{reinterpret_cast<const float*>(mf[m].b.F), rows, 1, 0, h.D, h.D, w3[m].wh(l, 0),
                                 w3[m].wh(l, 1), h.D, nullptr, 1, reinterpret_cast<float*>(mf[m].b.Z), h.D, 0, false};
          }
        }
        if (nj > 0) DQ_LAUNCH(H, kb + PK_GEMM_NODE, gemm_tf32x3_tc_jobs(jd, nj, H.d_status, s));
      }
      // molecules on the fused layer kernel (as in their single-molecule calls) leave the
      // grouped message, update-map and update launches
      MolFwd<T> rest[kMaxGroup];
      bool fused[kMaxGroup];
      for (int m = 0; m < n; ++m) {
        rest[m] = mf[m];
        fused[m] = use_fused(*g.h[m], jets) && mf[m].d.Bc > 0;
        if (fused[m]) rest[m].d.Bc = 0;
      }
      DQ_LAUNCH(H, kb + PK_MESSAGES, launch_messages_group<T>(rest, n, l, l == 0, s));
      nj = 0;
      for (int m = 0; m < n; ++m) {  // update map W_g [m_par; m_anti; m_nuc] + b_g
        const dq_handle_s& h = *g.h[m];
        const FwdDims& d = rest[m].d;
        if (d.Bc <= 0) continue;
        const int64_t rows = d.Bc * d.N * d.C;
        const float* bg = reinterpret_cast<const float*>(params[m] + h.off.layer[l].b_g);
        if (use_tc) {
          DQ_LAUNCH(H, kb + PK_GEMM_UPDATE,
                    gemm_bf16_tc(mf[m].b.msg_bf, rows, 3 * h.D, 3 * h.D, Wbf[m] + (size_t)l * 4 * h.D * h.D * 2, h.D,
                                 bg, d.C, reinterpret_cast<float*>(mf[m].b.Z), h.D, H.d_status, s));
        } else {
          jd[nj++] = T3JobDesc{reinterpret_cast<const float*>(mf[m].b.msg), rows, 1, 0, 3 * h.D, 3 * h.D,
                               w3[m].wg(l, 0), w3[m].wg(l, 1), h.D, bg, d.C, reinterpret_cast<float*>(mf[m].b.Z), h.D,
                               0, false};
        }
      }
      if (!use_tc) DQ_LAUNCH(H, kb + PK_GEMM_UPDATE, gemm_tf32x3_tc_jobs(jd, nj, H.d_status, s));
      DQ_LAUNCH(H, kb + PK_UPDATE, launch_update_group<T>(rest, n, l == 0, s));
      for (int m = 0; m < n; ++m)
        if (fused[m]) {
          const dq_handle_s& h = *g.h[m];
          const bool z_const = l == 0 && !h.el_init;
          DQ_LAUNCH(H, kb + PK_LAYER_FUSED,
                    launch_layer_fused(h, mf[m].d, params[m], l, z_const, mf[m].b.Z, mf[m].b.z0, mf[m].b.ew,
                                       mf[m].b.geo, mf[m].b.msg, w3[m].wg(l, 0), w3[m].wg(l, 1),
                                       use_tc ? Wbf[m] + (size_t)l * 4 * h.D * h.D * 2 : nullptr, s));
          FwdBuffers<T> bu = mf[m].b;
          bu.F_bf = nullptr;
          DQ_LAUNCH(H, kb + PK_UPDATE, launch_update<T>(h, mf[m].d, params[m], z_const, bu, s));
        }
    }
    int nj = 0;
    for (int m = 0; m < n; ++m) {  // orbitals of both spins of every molecule
      const dq_handle_s& h = *g.h[m];
      const FwdDims& d = mf[m].d;
      if (d.Bc <= 0) continue;
      const int Wo = h.K * h.det_n(), C = d.C, D = h.D, N = h.N;
      const int ns[2] = {h.n_up, h.n_dn}, i0[2] = {0, h.n_up};
      for (int sp = 0; sp < 2; ++sp)
        jd[nj++] = T3JobDesc{reinterpret_cast<const float*>(mf[m].b.F) + (int64_t)i0[sp] * C * D,
                             (int64_t)ns[sp] * C, d.Bc, (int64_t)N * C * D, D, D, w3[m].wo(sp, 0), w3[m].wo(sp, 1),
                             h.K * h.ncol(sp), reinterpret_cast<const float*>(params[m] + h.off.b_o[sp]), C,
                             reinterpret_cast<float*>(mf[m].b.phi) + (int64_t)i0[sp] * C * Wo, Wo,
                             (int64_t)N * C * Wo, false};
    }
    DQ_LAUNCH(H, kb + PK_GEMM_ORBITAL, gemm_tf32x3_tc_jobs(jd, nj, H.d_status, s));
    DQ_LAUNCH(H, kb + PK_ORBITAL_DET, launch_orbital_det_group<T>(mf, n, s));
    DQ_LAUNCH(H, kb + PK_JASTROW_SUM, launch_jastrow_sum_group<T>(mf, n, s));
    nj = 0;
    for (int m = 0; m < n; ++m) {
      const dq_handle_s& h = *g.h[m];
      const FwdDims& d = mf[m].d;
      if (d.Bc <= 0 || !h.use_jastrow) continue;
      jd[nj++] = T3JobDesc{reinterpret_cast<const float*>(mf[m].b.js), d.Bc * d.C, 1, 0, h.D, h.D, w3[m].wj(0),
                           w3[m].wj(1), h.D, reinterpret_cast<const float*>(params[m] + h.off.b_J1), d.C,
                           reinterpret_cast<float*>(mf[m].b.jh), h.D, 0, false};
    }
    DQ_LAUNCH(H, kb + PK_GEMM_JASTROW, gemm_tf32x3_tc_jobs(jd, nj, H.d_status, s));
    DQ_LAUNCH(H, kb + PK_COMBINE, launch_combine_group<T>(mf, n, la, sg, e_loc ? el : nullptr, nullptr, s));
  }
  return DQ_OK;
}

// Metropolis steps of a batch: one grouped proposal, value-only forward and
// accept launch per step; molecule m's draws equal mcmc_step's on its own handle.
struct MultiMcmcPlan {
  size_t r_prop[kMaxGroup], la_prop[kMaxGroup], sign_prop[kMaxGroup], fwd;
  MultiFwdPlan fp;
  size_t total;
};
MultiMcmcPlan plan_mcmc_multi(const dq_multi_s& g, const int64_t* B, size_t elem) {
  MultiMcmcPlan p{};
  size_t o = 0;
  for (int m = 0; m < g.n; ++m) {
    const size_t b = (size_t)std::max<int64_t>(B[m], 1);
    p.r_prop[m] = o;
    o += align_up(b * 3 * g.h[m]->N * elem);
    p.la_prop[m] = o;
    o += align_up(b * elem);
    p.sign_prop[m] = o;
    o += align_up(b);
  }
  p.fwd = o;
  p.fp = plan_forward_multi(g, B, false, elem);
  p.total = o + p.fp.total;
  return p;
}

template <class T>
dq_status run_mcmc_multi(const dq_multi_s& g, const T* const* params, T* const* r, T* const* logabs, const int64_t* B,
                         int32_t n_steps, double step, uint64_t seed, uint64_t t0, uint64_t* t_dev,
                         int64_t* const* n_acc, unsigned char* ws, size_t ws_bytes, cudaStream_t s) {
  const int n = g.n;
  const MultiMcmcPlan plan = plan_mcmc_multi(g, B, sizeof(T));
  if (ws == nullptr || ws_bytes < plan.total || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  const dq_handle_s& H = *g.h[0];
  T *rp[kMaxGroup], *lp[kMaxGroup];
  const T *rpc[kMaxGroup], *lpc[kMaxGroup], *rc[kMaxGroup];
  int8_t* sp[kMaxGroup];
  const int8_t* spc[kMaxGroup];
  unsigned long long* acc[kMaxGroup];
  const dq_handle_s* hs[kMaxGroup];
  for (int m = 0; m < n; ++m) {
    hs[m] = g.h[m];
    rp[m] = reinterpret_cast<T*>(ws + plan.r_prop[m]);
    lp[m] = reinterpret_cast<T*>(ws + plan.la_prop[m]);
    sp[m] = reinterpret_cast<int8_t*>(ws + plan.sign_prop[m]);
    rpc[m] = rp[m];
    lpc[m] = lp[m];
    spc[m] = sp[m];
    rc[m] = r[m];
    acc[m] = n_acc ? reinterpret_cast<unsigned long long*>(n_acc[m]) : nullptr;
    if (acc[m]) DQ_CU(cudaMemsetAsync(acc[m], 0, sizeof(int64_t), s));
  }
  for (int32_t k = 0; k < n_steps; ++k) {
    const uint64_t t = t0 + (uint64_t)k;
    DQ_LAUNCH(H, PK_PROPOSE, launch_propose_group<T>(hs, n, B, rc, rp, step, seed, t, t_dev, s));
    dq_status st = run_forward_multi<T>(g, params, rpc, B, false, lp, sp, nullptr, ws + plan.fwd, ws_bytes - plan.fwd,
                                        s, &plan.fp);
    if (st != DQ_OK) return st;
    DQ_LAUNCH(H, PK_ACCEPT, launch_accept_group<T>(hs, n, B, r, logabs, rpc, lpc, spc, seed, t, t_dev,
                                                   n_acc ? acc : nullptr, s));
  }
  if (t_dev && n_steps > 0) DQ_CU(launch_advance_counter(t_dev, (uint64_t)n_steps, s));
  return DQ_OK;
}

// Reverse pass of a batch: molecule by molecule (run_grad), each in its own
// workspace region.
struct MultiGradPlan {
  size_t off[kMaxGroup];
  size_t bytes[kMaxGroup];
  size_t total;
};
MultiGradPlan plan_grad_multi(const dq_multi_s& g, const int64_t* B, size_t elem) {
  MultiGradPlan p{};
  size_t o = 0;
  for (int m = 0; m < g.n; ++m) {
    const int64_t Bc = std::max<int64_t>(1, std::min<int64_t>(B[m], g.h[m]->max_chunk));
    p.off[m] = o;
    p.bytes[m] = plan_grad(*g.h[m], Bc, elem).total;
    o += align_up(p.bytes[m]);
  }
  p.total = o;
  return p;
}

size_t loss_scratch_multi(const dq_multi_s& g, const int64_t* B, size_t* off) {
  size_t o = 0;
  for (int m = 0; m < g.n; ++m) {
    if (off) off[m] = o;
    o += loss_scratch_bytes(std::max<int64_t>(B[m], 1));
  }
  return o;
}

// Autotuner workspace: the largest candidate's forward (one round), then the
// timing outputs (log|psi|, E_loc, sign of every molecule).
size_t autotune_bytes(dq_multi_s& g, const int64_t* B) {
  const int keep = g.rounds;
  g.rounds = 1;
  size_t o = plan_forward_multi(g, B, true, 4).total;
  g.rounds = keep;
  for (int m = 0; m < g.n; ++m) o += 2 * align_up((size_t)std::max<int64_t>(B[m], 1) * 4) + align_up((size_t)std::max<int64_t>(B[m], 1));
  return o;
}

dq_status check_multi(dq_multi g) {
  if (g == nullptr) return DQ_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return DQ_ERR_CUDA;
  if (dev != g->device) return DQ_ERR_ARG;
  return DQ_OK;
}
// Pseudopotential energies: displaced configurations, their value-only forward, the
// quadrature sums (pseudo.cu).
struct PPPlan {
  int64_t nconf;
  size_t configs, la, sg, fwd, total;
};
PPPlan plan_pp(const dq_handle_s& h, int64_t B, int n_pp, size_t elem) {
  PPPlan p{};
  p.nconf = B * h.N * n_pp * 12;
  size_t o = 0;
  p.configs = o;
  o += align_up((size_t)p.nconf * h.N * 3 * elem);
  p.la = o;
  o += align_up((size_t)p.nconf * elem);
  p.sg = o;
  o += align_up((size_t)p.nconf);
  p.fwd = o;
  o += plan_forward(h, std::max<int64_t>(1, std::min<int64_t>(p.nconf, h.max_chunk)), false, elem).total;
  p.total = o;
  return p;
}

template <class T>
dq_status run_pp(const dq_handle_s& h, const T* params, const T* r, int64_t B, const PPSet& pp, const T* rot,
                 const T* logabs, const int8_t* sign, T* v_loc, T* v_nl, unsigned char* ws, size_t ws_bytes,
                 cudaStream_t s) {
  const PPPlan plan = plan_pp(h, B, pp.n, sizeof(T));
  if (!ws || ws_bytes < plan.total || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  T* configs = reinterpret_cast<T*>(ws + plan.configs);
  T* la = reinterpret_cast<T*>(ws + plan.la);
  int8_t* sg = reinterpret_cast<int8_t*>(ws + plan.sg);
  DQ_CU(pp_displace<T>(r, h.d_R, rot, B, h.N, pp, configs, s));
  const dq_status st = run_forward<T>(h, params, configs, plan.nconf, false, la, sg, nullptr, ws + plan.fwd,
                                      ws_bytes - plan.fwd, s);
  if (st != DQ_OK) return st;
  DQ_CU(pp_combine<T>(r, h.d_R, rot, logabs, sign, la, sg, B, h.N, pp, v_loc, v_nl, s));
  return DQ_OK;
}

dq_status make_ppset(const dq_handle_s& h, int32_t n_pp, const dq_pseudopotential* pps, PPSet* out) {
  if (n_pp < 1 || n_pp > kMaxPP || !pps) return DQ_ERR_ARG;
  PPSet& p = *out;
  p = PPSet{};
  p.n = n_pp;
  for (int q = 0; q < n_pp; ++q) {
    const dq_pseudopotential& d = pps[q];
    if (d.nucleus < 0 || d.nucleus >= h.M || d.l_max < 0 || d.l_max > kMaxPPChan - 2 || d.n_terms < 1 ||
        d.n_terms > kMaxPPTerms || !d.coef)
      return DQ_ERR_ARG;
    p.nucleus[q] = d.nucleus;
    p.lmax[q] = d.l_max;
    p.n_terms[q] = d.n_terms;
    for (int c = 0; c < d.l_max + 2; ++c)
      for (int t = 0; t < d.n_terms; ++t)
        for (int x = 0; x < 3; ++x) {
          const double v = d.coef[(c * d.n_terms + t) * 3 + x];
          if (!isfinite(v)) return DQ_ERR_ARG;
          p.c[(q * kMaxPPChan + c) * kMaxPPTerms + t][x] = v;
        }
  }
  return DQ_OK;
}
}  // namespace
}  // namespace dq

using namespace dq;

extern "C" {

const char* dq_status_string(dq_status s) {
  switch (s) {
    case DQ_OK: return "ok";
    case DQ_ERR_ARG: return "invalid argument";
    case DQ_ERR_SHAPE: return "unsupported shape";
    case DQ_ERR_CUDA: return "CUDA error";
    case DQ_ERR_NONFINITE: return "non-finite result";
    case DQ_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case DQ_ERR_TIMEOUT: return "device wait timed out";
    case DQ_ERR_UNSUPPORTED: return "unsupported in this precision";
  }
  return "unknown status";
}

dq_status dq_create(const dq_system* sys, const dq_ansatz_cfg* cfg, int32_t precision, dq_handle* out) {
  if (!sys || !cfg || !out) return DQ_ERR_ARG;
  *out = nullptr;
  if (precision != DQ_FP64 && precision != DQ_FP32 && precision != DQ_BF16_MIXED) return DQ_ERR_ARG;
  if (!sys->Z || !sys->R) return DQ_ERR_ARG;
  const int M = sys->n_nuc, n_up = sys->n_up, n_dn = sys->n_down, N = n_up + n_dn;
  if (M < 1 || M > kMaxNuc || n_up < 1 || n_dn < 0 || N > kMaxElec || n_up > kMaxSpin || n_dn > kMaxSpin)
    return DQ_ERR_SHAPE;
  if (cfg->width < 32 || cfg->width % 32 || cfg->width > 512 || cfg->n_layers < 1 || cfg->n_layers > kMaxLayers ||
      cfg->n_det < 1 || cfg->n_det > 128 || cfg->n_rbf < 8 || cfg->n_rbf % 8 || cfg->n_rbf > 64 ||
      !(cfg->rbf_cutoff > 0) || !(cfg->cusp_alpha > 0))
    return DQ_ERR_SHAPE;
  // the BF16 tensor-core GEMMs take K = D and 3D in 64-wide tiles
  if (precision == DQ_BF16_MIXED && cfg->width % 64) return DQ_ERR_SHAPE;
  if (cfg->full_det != 0 && cfg->full_det != 1) return DQ_ERR_ARG;
  if (cfg->edge_update != 0 && cfg->edge_update != 1) return DQ_ERR_ARG;
  if (cfg->el_init != 0 && cfg->el_init != 1) return DQ_ERR_ARG;
  if (cfg->full_det && N > kMaxSpin) return DQ_ERR_SHAPE;  // the N x N matrix obeys the spin-block limit
  for (int I = 0; I < M; ++I) {
    if (!isfinite(sys->Z[I])) return DQ_ERR_ARG;
    for (int x = 0; x < 3; ++x)
      if (!isfinite(sys->R[3 * I + x])) return DQ_ERR_ARG;
  }
  dq_handle_s* h = new (std::nothrow) dq_handle_s();
  if (!h) return DQ_ERR_ARG;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return DQ_ERR_CUDA;
  }
  h->precision = precision;
  h->n_up = n_up;
  h->n_dn = n_dn;
  h->N = N;
  h->M = M;
  h->D = cfg->width;
  h->L = cfg->n_layers;
  h->K = cfg->n_det;
  h->Q = cfg->n_rbf;
  h->rc = cfg->rbf_cutoff;
  h->alpha = cfg->cusp_alpha;
  h->use_jastrow = cfg->use_jastrow ? 1 : 0;
  h->use_cusp = cfg->use_cusp ? 1 : 0;
  h->full_det = cfg->full_det;
  h->edge_update = cfg->edge_update;
  h->el_init = cfg->el_init;
  h->off = make_offsets(h->D, h->L, h->K, h->Q, M, h->ncol(0), h->ncol(1), h->edge_update, h->el_init);
  double vnn = 0;
  for (int I = 0; I < M; ++I)
    for (int J = I + 1; J < M; ++J) {
      double d2 = 0;
      for (int x = 0; x < 3; ++x) d2 += (sys->R[3 * I + x] - sys->R[3 * J + x]) * (sys->R[3 * I + x] - sys->R[3 * J + x]);
      vnn += sys->Z[I] * sys->Z[J] / sqrt(d2);
    }
  h->Vnn = vnn;
  // Edge tables: same-spin pairs (up-up, then down-down), opposite-spin pairs.
  std::vector<int> pij, pof(N * N, -1);
  auto add = [&](int i, int j) {
    pof[i * N + j] = pof[j * N + i] = (int)(pij.size() / 2);
    pij.push_back(i);
    pij.push_back(j);
  };
  for (int i = 0; i < n_up; ++i)
    for (int j = i + 1; j < n_up; ++j) add(i, j);
  for (int i = n_up; i < N; ++i)
    for (int j = i + 1; j < N; ++j) add(i, j);
  const int n_par = (int)pij.size() / 2;
  for (int i = 0; i < n_up; ++i)
    for (int j = n_up; j < N; ++j) add(i, j);
  h->edges.n_par = n_par;
  h->edges.n_ee = (int)pij.size() / 2;
  h->edges.n_anti = h->edges.n_ee - n_par;
  h->edges.n_en = N * M;
  h->edges.n_all = h->edges.n_ee + h->edges.n_en;
  if (pij.empty()) pij.assign(2, 0);
  std::vector<float> Rf(3 * M);
  for (int k = 0; k < 3 * M; ++k) Rf[k] = (float)sys->R[k];
  bool ok = cudaMalloc(&h->d_R, 3 * M * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->d_Rf, 3 * M * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&h->d_Z, M * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->d_pair_of, N * N * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->d_pair_ij, pij.size() * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->d_status, sizeof(unsigned int)) == cudaSuccess &&
            cudaMalloc(&h->d_fp64_count, sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMemcpy(h->d_R, sys->R, 3 * M * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(h->d_Rf, Rf.data(), 3 * M * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(h->d_Z, sys->Z, M * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(h->d_pair_of, pof.data(), N * N * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(h->d_pair_ij, pij.data(), pij.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(h->d_status, 0, sizeof(unsigned int)) == cudaSuccess &&
       cudaMemset(h->d_fp64_count, 0, sizeof(unsigned long long)) == cudaSuccess;
  if (!ok) {
    dq_destroy(h);
    return DQ_ERR_CUDA;
  }
  *out = h;
  return DQ_OK;
}

dq_status dq_destroy(dq_handle h) {
  if (!h) return DQ_ERR_ARG;
  cudaFree(h->d_R);
  cudaFree(h->d_Rf);
  cudaFree(h->d_Z);
  cudaFree(h->d_pair_of);
  cudaFree(h->d_pair_ij);
  cudaFree(h->d_status);
  cudaFree(h->d_fp64_count);
  if (h->prof) {
    for (cudaEvent_t e : h->prof->pool) cudaEventDestroy(e);
    delete h->prof;
  }
  delete h;
  return DQ_OK;
}

dq_status dq_param_count(dq_handle h, int64_t* P) {
  if (!h || !P) return DQ_ERR_ARG;
  *P = h->off.total;
  return DQ_OK;
}

dq_status dq_max_chunk(dq_handle h, int64_t* chunk) {
  if (!h || !chunk) return DQ_ERR_ARG;
  *chunk = h->max_chunk;
  return DQ_OK;
}

dq_status dq_set_max_chunk(dq_handle h, int64_t chunk) {
  if (!h || chunk < 1) return DQ_ERR_ARG;
  h->max_chunk = chunk;
  return DQ_OK;
}

dq_status dq_workspace_size(dq_handle h, int64_t B, int32_t op, size_t* bytes) {
  if (!h || !bytes || B < 0) return DQ_ERR_ARG;
  const int64_t Bc = std::max<int64_t>(1, std::min<int64_t>(B, h->max_chunk));
  const size_t el = elem_size(*h);
  switch (op) {
    case DQ_OP_EVAL: *bytes = plan_forward(*h, Bc, false, el).total; return DQ_OK;
    case DQ_OP_LOCAL_ENERGY: *bytes = plan_forward(*h, Bc, true, el).total; return DQ_OK;
    case DQ_OP_MCMC: *bytes = plan_mcmc(*h, std::max<int64_t>(B, 1), el).total; return DQ_OK;
    case DQ_OP_GRAD: *bytes = plan_grad(*h, Bc, el).total; return DQ_OK;
    case DQ_OP_LOSS_WEIGHTS: *bytes = loss_scratch_bytes(std::max<int64_t>(B, 1)); return DQ_OK;
    case DQ_OP_MALA: *bytes = plan_mala(*h, std::max<int64_t>(B, 1), el).total; return DQ_OK;
    case DQ_OP_NATGRAD: *bytes = natgrad_workspace(std::max<int64_t>(B, 2), h->off.total); return DQ_OK;
    case DQ_OP_UPDATE: *bytes = param_update_workspace(); return DQ_OK;
  }
  return DQ_ERR_ARG;
}

dq_status ansatz_eval(dq_handle h, const void* params, const void* r, int64_t B, void* logabs, int8_t* sign, void* ws,
                      size_t ws_bytes, void* stream) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (B < 0) return DQ_ERR_ARG;
  if (B == 0) return DQ_OK;
  if (!params || !r || !logabs || !sign) return DQ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  auto* w = static_cast<unsigned char*>(ws);
  if (h->precision == DQ_FP64)
    return run_forward<double>(*h, (const double*)params, (const double*)r, B, false, (double*)logabs, sign, nullptr,
                               w, ws_bytes, s);
  return run_forward<float>(*h, (const float*)params, (const float*)r, B, false, (float*)logabs, sign, nullptr, w,
                            ws_bytes, s);
}

dq_status local_energy(dq_handle h, const void* params, const void* r, int64_t B, void* logabs, int8_t* sign,
                       void* e_loc, double* e_sum2, void* ws, size_t ws_bytes, void* stream) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (B < 0) return DQ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (B == 0) {
    if (e_sum2 && cudaMemsetAsync(e_sum2, 0, 2 * sizeof(double), s) != cudaSuccess) return DQ_ERR_CUDA;
    return DQ_OK;
  }
  if (!params || !r || !logabs || !sign || !e_loc) return DQ_ERR_ARG;
  auto* w = static_cast<unsigned char*>(ws);
  if (h->precision == DQ_FP64) {
    st = run_forward<double>(*h, (const double*)params, (const double*)r, B, true, (double*)logabs, sign,
                             (double*)e_loc, w, ws_bytes, s);
    if (st == DQ_OK && e_sum2) DQ_LAUNCH(*h, PK_ESUM, launch_esum<double>((const double*)e_loc, B, e_sum2, h->d_status, s));
  } else {
    st = run_forward<float>(*h, (const float*)params, (const float*)r, B, true, (float*)logabs, sign, (float*)e_loc,
                            w, ws_bytes, s);
    if (st == DQ_OK && e_sum2) DQ_LAUNCH(*h, PK_ESUM, launch_esum<float>((const float*)e_loc, B, e_sum2, h->d_status, s));
  }
  return st;
}


namespace {
dq_status mcmc_impl(dq_handle h, const void* params, void* r, void* logabs, int64_t B, int32_t n_steps,
                    double step_size, uint64_t seed, uint64_t step_counter, uint64_t* t_dev, int64_t* n_accepted,
                    void* ws, size_t ws_bytes, void* stream) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (B < 0 || n_steps < 0 || !(step_size >= 0) || !isfinite(step_size)) return DQ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (B == 0 || n_steps == 0) {
    if (n_accepted && cudaMemsetAsync(n_accepted, 0, sizeof(int64_t), s) != cudaSuccess) return DQ_ERR_CUDA;
    if (t_dev && n_steps > 0 && launch_advance_counter(t_dev, (uint64_t)n_steps, s) != cudaSuccess)
      return DQ_ERR_CUDA;
    return DQ_OK;
  }
  if (!params || !r || !logabs) return DQ_ERR_ARG;
  auto* w = static_cast<unsigned char*>(ws);
  if (h->precision == DQ_FP64)
    return run_mcmc<double>(h, (const double*)params, (double*)r, (double*)logabs, B, n_steps, step_size, seed,
                            step_counter, t_dev, n_accepted, w, ws_bytes, s);
  return run_mcmc<float>(h, (const float*)params, (float*)r, (float*)logabs, B, n_steps, step_size, seed,
                         step_counter, t_dev, n_accepted, w, ws_bytes, s);
}
}  // namespace

dq_status mcmc_step(dq_handle h, const void* params, void* r, void* logabs, int64_t B, int32_t n_steps,
                    double step_size, uint64_t seed, uint64_t step_counter, int64_t* n_accepted, void* ws,
                    size_t ws_bytes, void* stream) {
  return mcmc_impl(h, params, r, logabs, B, n_steps, step_size, seed, step_counter, nullptr, n_accepted, ws, ws_bytes,
                   stream);
}

dq_status mala_step(dq_handle h, const void* params, void* r, void* logabs, void* grad, void* e_loc,
                    int32_t grad_valid, int64_t B, int32_t n_steps, double tau, uint64_t seed, uint64_t step_counter,
                    uint64_t* step_counter_dev, int64_t* n_accepted, void* ws, size_t ws_bytes, void* stream) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (B < 0 || n_steps < 0 || !(tau > 0) || !isfinite(tau)) return DQ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (B == 0 || (n_steps == 0 && grad_valid)) {
    if (n_accepted && cudaMemsetAsync(n_accepted, 0, sizeof(int64_t), s) != cudaSuccess) return DQ_ERR_CUDA;
    if (step_counter_dev && n_steps > 0 && launch_advance_counter(step_counter_dev, (uint64_t)n_steps, s) != cudaSuccess)
      return DQ_ERR_CUDA;
    return DQ_OK;
  }
  if (!params || !r || !logabs || !grad) return DQ_ERR_ARG;
  auto* w = static_cast<unsigned char*>(ws);
  if (h->precision == DQ_FP64)
    return run_mala<double>(h, (const double*)params, (double*)r, (double*)logabs, (double*)grad, (double*)e_loc,
                            grad_valid, B, n_steps, tau, seed, step_counter, step_counter_dev, n_accepted, w, ws_bytes,
                            s);
  return run_mala<float>(h, (const float*)params, (float*)r, (float*)logabs, (float*)grad, (float*)e_loc, grad_valid, B,
                         n_steps, tau, seed, step_counter, step_counter_dev, n_accepted, w, ws_bytes, s);
}

dq_status mcmc_step_eloc(dq_handle h, const void* params, void* r, void* logabs, void* e_loc, int64_t B,
                         int32_t n_steps, double step_size, uint64_t seed, uint64_t step_counter,
                         uint64_t* step_counter_dev, int64_t* n_accepted, void* ws, size_t ws_bytes, void* stream) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (B < 0 || n_steps < 0 || !(step_size >= 0) || !isfinite(step_size)) return DQ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (B == 0 || n_steps == 0) {
    if (n_accepted && cudaMemsetAsync(n_accepted, 0, sizeof(int64_t), s) != cudaSuccess) return DQ_ERR_CUDA;
    if (step_counter_dev && n_steps > 0 && launch_advance_counter(step_counter_dev, (uint64_t)n_steps, s) != cudaSuccess)
      return DQ_ERR_CUDA;
    return DQ_OK;
  }
  if (!params || !r || !logabs || !e_loc) return DQ_ERR_ARG;
  auto* w = static_cast<unsigned char*>(ws);
  if (h->precision == DQ_FP64)
    return run_mcmc_eloc<double>(h, (const double*)params, (double*)r, (double*)logabs, (double*)e_loc, B, n_steps,
                                 step_size, seed, step_counter, step_counter_dev, n_accepted, w, ws_bytes, s);
  return run_mcmc_eloc<float>(h, (const float*)params, (float*)r, (float*)logabs, (float*)e_loc, B, n_steps,
                              step_size, seed, step_counter, step_counter_dev, n_accepted, w, ws_bytes, s);
}

dq_status mcmc_step_dev(dq_handle h, const void* params, void* r, void* logabs, int64_t B, int32_t n_steps,
                        double step_size, uint64_t seed, uint64_t* step_counter, int64_t* n_accepted, void* ws,
                        size_t ws_bytes, void* stream) {
  if (step_counter == nullptr) return DQ_ERR_ARG;
  return mcmc_impl(h, params, r, logabs, B, n_steps, step_size, seed, 0, step_counter, n_accepted, ws, ws_bytes,
                   stream);
}

dq_status grad_logpsi(dq_handle h, const void* params, const void* r, int64_t B, const void* weights, int32_t mode,
                      void* grad_out, void* ws, size_t ws_bytes, void* stream) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (B < 0 || (mode != 0 && mode != 1)) return DQ_ERR_ARG;
  if (!params || !grad_out || (B > 0 && !r) || (mode == 0 && B > 0 && !weights)) return DQ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t el = elem_size(*h);
  if (B == 0) {
    if (mode == 0 && cudaMemsetAsync(grad_out, 0, (size_t)h->off.total * el, s) != cudaSuccess) return DQ_ERR_CUDA;
    return DQ_OK;
  }
  auto* w = static_cast<unsigned char*>(ws);
  const void* wt = mode == 0 ? weights : nullptr;
  if (h->precision == DQ_FP64)
    return run_grad<double>(*h, (const double*)params, (const double*)r, B, (const double*)wt, mode, (double*)grad_out,
                            w, ws_bytes, s);
  return run_grad<float>(*h, (const float*)params, (const float*)r, B, (const float*)wt, mode, (float*)grad_out, w,
                         ws_bytes, s);
}

dq_status natural_gradient(dq_handle h, const void* G, const void* w, int64_t B, double lambda, int32_t max_iter,
                           double tol, void* delta, double* stats, void* ws, size_t ws_bytes, void* stream) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (h->precision == DQ_FP64) return DQ_ERR_UNSUPPORTED;
  if (!G || !w || !delta || B < 2 || lambda == 0 || !isfinite(lambda) || max_iter < 0 || !(tol >= 0))
    return DQ_ERR_ARG;
  if (B > (int64_t)INT32_MAX || h->off.total > (int64_t)INT32_MAX) return DQ_ERR_SHAPE;
  if (!ws || ws_bytes < natgrad_workspace(B, h->off.total) || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  const cudaError_t e = natgrad_run(static_cast<const float*>(G), static_cast<const float*>(w), B, h->off.total,
                                    lambda, max_iter, tol, static_cast<float*>(delta), stats,
                                    static_cast<unsigned char*>(ws), h->d_status, (cudaStream_t)stream);
  if (e == cudaErrorInvalidValue) return DQ_ERR_ARG;
  return e == cudaSuccess ? DQ_OK : DQ_ERR_CUDA;
}

dq_status param_update(dq_handle h, void* params, const void* delta, double lr, double max_norm, double* stats,
                       void* ws, size_t ws_bytes, void* stream) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (h->precision == DQ_FP64) return DQ_ERR_UNSUPPORTED;
  if (!params || !delta || !stats || !isfinite(lr) || !isfinite(max_norm)) return DQ_ERR_ARG;
  if (!ws || ws_bytes < param_update_workspace() || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  const cudaError_t e = param_update_run<float>(static_cast<float*>(params), static_cast<const float*>(delta),
                                                h->off.total, lr, max_norm, stats, static_cast<unsigned char*>(ws),
                                                (cudaStream_t)stream);
  return e == cudaSuccess ? DQ_OK : DQ_ERR_CUDA;
}

dq_status dq_pp_workspace_size(dq_handle h, int64_t B, int32_t n_pp, size_t* bytes) {
  if (!h || !bytes || B < 0 || n_pp < 1 || n_pp > kMaxPP) return DQ_ERR_ARG;
  *bytes = plan_pp(*h, std::max<int64_t>(B, 1), n_pp, elem_size(*h)).total;
  return DQ_OK;
}

dq_status pseudopotential_energy(dq_handle h, const void* params, const void* r, int64_t B, int32_t n_pp,
                                 const dq_pseudopotential* pps, const void* rot, const void* logabs,
                                 const int8_t* sign, void* v_loc, void* v_nl, void* ws, size_t ws_bytes,
                                 void* stream) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (B < 0) return DQ_ERR_ARG;
  if (B == 0) return DQ_OK;
  if (!params || !r || !rot || !logabs || !sign || !v_loc || !v_nl) return DQ_ERR_ARG;
  PPSet pp;
  st = make_ppset(*h, n_pp, pps, &pp);
  if (st != DQ_OK) return st;
  auto* w = static_cast<unsigned char*>(ws);
  const cudaStream_t s = (cudaStream_t)stream;
  if (h->precision == DQ_FP64)
    return run_pp<double>(*h, (const double*)params, (const double*)r, B, pp, (const double*)rot,
                          (const double*)logabs, sign, (double*)v_loc, (double*)v_nl, w, ws_bytes, s);
  return run_pp<float>(*h, (const float*)params, (const float*)r, B, pp, (const float*)rot, (const float*)logabs,
                       sign, (float*)v_loc, (float*)v_nl, w, ws_bytes, s);
}

dq_status vmc_loss_weights_clip(dq_handle h, const void* e_loc, int64_t B, double clip_k, int32_t clip_mode,
                                void* weights, double* stats, void* ws, size_t ws_bytes, void* stream) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (B < 1 || B > 65536 || !e_loc || !weights || !(clip_k > 0)) return DQ_ERR_ARG;
  if (clip_mode != DQ_CLIP_HARD && clip_mode != DQ_CLIP_LOG) return DQ_ERR_ARG;
  if (!ws || ws_bytes < loss_scratch_bytes(B) || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const int soft = clip_mode == DQ_CLIP_LOG ? 1 : 0;
  if (h->precision == DQ_FP64)
    DQ_LAUNCH(*h, PK_LOSS_WEIGHTS, launch_loss_weights<double>((const double*)e_loc, B, clip_k, (double*)weights, stats, (double*)ws, s, soft));
  else
    DQ_LAUNCH(*h, PK_LOSS_WEIGHTS, launch_loss_weights<float>((const float*)e_loc, B, clip_k, (float*)weights, stats, (double*)ws, s, soft));
  return DQ_OK;
}

dq_status vmc_loss_weights(dq_handle h, const void* e_loc, int64_t B, double clip_k, void* weights, double* stats,
                           void* ws, size_t ws_bytes, void* stream) {
  return vmc_loss_weights_clip(h, e_loc, B, clip_k, DQ_CLIP_HARD, weights, stats, ws, ws_bytes, stream);
}

dq_status dq_last_device_status(dq_handle h, void* stream, uint32_t* flags) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (!flags) return DQ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned int v = 0;
  DQ_CU(cudaMemcpyAsync(&v, h->d_status, sizeof(v), cudaMemcpyDeviceToHost, s));
  DQ_CU(cudaStreamSynchronize(s));
  DQ_CU(cudaMemsetAsync(h->d_status, 0, sizeof(v), s));
  *flags = v;
  return DQ_OK;
}

dq_status dq_profile_enable(dq_handle h, int32_t on) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (!h->prof) {
    h->prof = new (std::nothrow) Profiler();
    if (!h->prof) return DQ_ERR_ARG;
  }
  if (on && h->prof->pool.empty()) {
    h->prof->pool.resize(1 << 15);
    for (auto& e : h->prof->pool)
      if (cudaEventCreate(&e) != cudaSuccess) return DQ_ERR_CUDA;
  }
  h->prof->on = on != 0;
  return DQ_OK;
}

dq_status dq_profile_reset(dq_handle h) {
  if (!h) return DQ_ERR_ARG;
  if (h->prof) {
    h->prof->kinds.clear();
    h->prof->next = 0;
    h->prof->overflow = false;
  }
  return DQ_OK;
}

dq_status dq_profile_read(dq_handle h, int32_t kind, double* total_ms, int64_t* launches) {
  if (!h || !total_ms || !launches || kind < 0 || kind >= PK_COUNT) return DQ_ERR_ARG;
  *total_ms = 0;
  *launches = 0;
  if (!h->prof) return DQ_OK;
  Profiler& p = *h->prof;
  for (size_t r = 0; r < p.kinds.size(); ++r) {
    if (p.kinds[r] != kind || 2 * r + 1 >= p.next) continue;
    if (cudaEventSynchronize(p.pool[2 * r + 1]) != cudaSuccess) return DQ_ERR_CUDA;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.pool[2 * r], p.pool[2 * r + 1]) != cudaSuccess) return DQ_ERR_CUDA;
    *total_ms += ms;
    *launches += 1;
  }
  return p.overflow ? DQ_ERR_WORKSPACE : DQ_OK;
}

const char* dq_profile_kind_name(int32_t kind) { return prof_kind_name(kind); }

dq_status dq_fp64_matrix_count(dq_handle h, void* stream, int64_t* count) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (!count) return DQ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long v = 0;
  DQ_CU(cudaMemcpyAsync(&v, h->d_fp64_count, sizeof(v), cudaMemcpyDeviceToHost, s));
  DQ_CU(cudaStreamSynchronize(s));
  DQ_CU(cudaMemsetAsync(h->d_fp64_count, 0, sizeof(v), s));
  *count = (int64_t)v;
  return DQ_OK;
}

int32_t dq_profile_kind_count(void) { return PK_COUNT; }

dq_status dq_test_gemm_bf16(const void* X, int64_t rows, int32_t K, int64_t ldx, const void* W, int32_t n_out,
                            const float* bias, int32_t bias_period, float* Y, int64_t ldy, uint32_t* status,
                            void* stream) {
  if (!X || !W || !Y || !status || rows < 0 || n_out < 0 || ldy < n_out) return DQ_ERR_ARG;
  const cudaError_t e = gemm_bf16_tc(X, rows, K, ldx, W, n_out, bias, bias_period, Y, ldy, status,
                                     (cudaStream_t)stream);
  if (e == cudaErrorInvalidValue) return DQ_ERR_ARG;
  return e == cudaSuccess ? DQ_OK : DQ_ERR_CUDA;
}

dq_status dq_test_gemm_tf32x3(const float* X, int64_t rows, int32_t K, int64_t ldx, const float* W, int32_t n_out,
                              const float* bias, int32_t bias_period, float* Y, int64_t ldy, float* wsplit,
                              uint32_t* status, void* stream) {
  if (!X || !W || !Y || !wsplit || !status || rows < 0 || n_out < 0 || K <= 0 || ldy < n_out) return DQ_ERR_ARG;
  const cudaStream_t s = (cudaStream_t)stream;
  const int64_t nw = (int64_t)n_out * K;
  cudaError_t e = split_tf32(W, wsplit, wsplit + nw, nw, s);
  if (e == cudaSuccess)
    e = gemm_tf32x3_tc(X, rows, K, ldx, wsplit, wsplit + nw, n_out, bias, bias_period, Y, ldy, status, s);
  if (e == cudaErrorInvalidValue) return DQ_ERR_ARG;
  return e == cudaSuccess ? DQ_OK : DQ_ERR_CUDA;
}

// ---- batches of molecules ----
dq_status dq_create_multi(int32_t n_mol, const dq_system* systems, const dq_ansatz_cfg* cfgs, int32_t precision,
                          dq_multi* out) {
  if (!out || !systems || !cfgs) return DQ_ERR_ARG;
  *out = nullptr;
  if (n_mol < 1 || n_mol > DQ_MAX_BATCH || DQ_MAX_BATCH > kMaxGroup) return DQ_ERR_SHAPE;
  if (precision == DQ_FP64) return DQ_ERR_UNSUPPORTED;
  if (precision != DQ_FP32 && precision != DQ_BF16_MIXED) return DQ_ERR_ARG;
  for (int m = 0; m < n_mol; ++m)
    if (cfgs[m].n_layers != cfgs[0].n_layers || cfgs[m].width % 32) return DQ_ERR_SHAPE;
  dq_multi_s* g = new (std::nothrow) dq_multi_s();
  if (!g) return DQ_ERR_ARG;
  if (cudaGetDevice(&g->device) != cudaSuccess) {
    delete g;
    return DQ_ERR_CUDA;
  }
  g->precision = precision;
  for (int m = 0; m < n_mol; ++m) {
    dq_handle h = nullptr;
    const dq_status st = dq_create(&systems[m], &cfgs[m], precision, &h);
    if (st != DQ_OK) {
      dq_destroy_multi(g);
      return st;
    }
    g->h[g->n++] = h;
  }
  *out = g;
  return DQ_OK;
}

dq_status dq_destroy_multi(dq_multi g) {
  if (!g) return DQ_ERR_ARG;
  dq_status st = DQ_OK;
  for (int m = 0; m < g->n; ++m)
    if (dq_destroy(g->h[m]) != DQ_OK) st = DQ_ERR_CUDA;
  delete g;
  return st;
}

dq_status dq_multi_handle(dq_multi g, int32_t k, dq_handle* h) {
  if (!g || !h || k < 0 || k >= g->n) return DQ_ERR_ARG;
  *h = g->h[k];
  return DQ_OK;
}

dq_status dq_multi_set_rounds(dq_multi g, int32_t rounds) {
  if (!g || rounds < 0) return DQ_ERR_ARG;
  g->rounds = rounds;
  return DQ_OK;
}

dq_status dq_multi_rounds(dq_multi g, int32_t* rounds) {
  if (!g || !rounds) return DQ_ERR_ARG;
  *rounds = g->rounds;
  return DQ_OK;
}

dq_status dq_multi_workspace_size(dq_multi g, const int64_t* B, int32_t op, size_t* bytes) {
  if (!g || !B || !bytes) return DQ_ERR_ARG;
  for (int m = 0; m < g->n; ++m)
    if (B[m] < 0) return DQ_ERR_ARG;
  const size_t el = 4;
  switch (op) {
    case DQ_OP_EVAL: *bytes = plan_forward_multi(*g, B, false, el).total; return DQ_OK;
    case DQ_OP_LOCAL_ENERGY: *bytes = plan_forward_multi(*g, B, true, el).total; return DQ_OK;
    case DQ_OP_MCMC: *bytes = plan_mcmc_multi(*g, B, el).total; return DQ_OK;
    case DQ_OP_GRAD: *bytes = plan_grad_multi(*g, B, el).total; return DQ_OK;
    case DQ_OP_LOSS_WEIGHTS: *bytes = loss_scratch_multi(*g, B, nullptr); return DQ_OK;
    case DQ_OP_AUTOTUNE: *bytes = autotune_bytes(*g, B); return DQ_OK;
  }
  return DQ_ERR_ARG;
}

namespace {
dq_status multi_args(dq_multi g, const int64_t* B, std::initializer_list<const void*> arrays) {
  dq_status st = check_multi(g);
  if (st != DQ_OK) return st;
  if (!B) return DQ_ERR_ARG;
  for (const void* a : arrays)
    if (!a) return DQ_ERR_ARG;
  for (int m = 0; m < g->n; ++m)
    if (B[m] < 0) return DQ_ERR_ARG;
  return DQ_OK;
}
// every molecule with walkers has its pointer in the host array arr
bool entries_set(const void* arr, const int64_t* B, int n) {
  const void* const* a = static_cast<const void* const*>(arr);
  for (int m = 0; m < n; ++m)
    if (B[m] > 0 && !a[m]) return false;
  return true;
}
}  // namespace

dq_status ansatz_eval_multi(dq_multi g, const void* const* params, const void* const* r, const int64_t* B,
                            void* const* logabs, int8_t* const* sign, void* ws, size_t ws_bytes, void* stream) {
  dq_status st = multi_args(g, B, {params, r, logabs, sign});
  if (st != DQ_OK) return st;
  if (!entries_set(params, B, g->n) || !entries_set(r, B, g->n) || !entries_set(logabs, B, g->n) ||
      !entries_set(sign, B, g->n))
    return DQ_ERR_ARG;
  return run_forward_multi<float>(*g, reinterpret_cast<const float* const*>(params),
                                  reinterpret_cast<const float* const*>(r), B, false,
                                  reinterpret_cast<float* const*>(logabs), sign, nullptr,
                                  static_cast<unsigned char*>(ws), ws_bytes, (cudaStream_t)stream);
}

dq_status local_energy_multi(dq_multi g, const void* const* params, const void* const* r, const int64_t* B,
                             void* const* logabs, int8_t* const* sign, void* const* e_loc, double* const* e_sum2,
                             void* ws, size_t ws_bytes, void* stream) {
  dq_status st = multi_args(g, B, {params, r, logabs, sign, e_loc});
  if (st != DQ_OK) return st;
  if (!entries_set(params, B, g->n) || !entries_set(r, B, g->n) || !entries_set(logabs, B, g->n) ||
      !entries_set(sign, B, g->n) || !entries_set(e_loc, B, g->n))
    return DQ_ERR_ARG;
  const cudaStream_t s = (cudaStream_t)stream;
  st = run_forward_multi<float>(*g, reinterpret_cast<const float* const*>(params),
                                reinterpret_cast<const float* const*>(r), B, true,
                                reinterpret_cast<float* const*>(logabs), sign, reinterpret_cast<float* const*>(e_loc),
                                static_cast<unsigned char*>(ws), ws_bytes, s);
  if (st != DQ_OK || !e_sum2) return st;
  double* out2[kMaxGroup];
  unsigned int* status[kMaxGroup];
  for (int m = 0; m < g->n; ++m) {
    out2[m] = e_sum2[m];
    status[m] = g->h[m]->d_status;
    if (out2[m] && B[m] == 0) DQ_CU(cudaMemsetAsync(out2[m], 0, 2 * sizeof(double), s));
    if (B[m] == 0) out2[m] = nullptr;
  }
  DQ_LAUNCH(*g->h[0], PK_ESUM, launch_esum_group<float>(g->n, reinterpret_cast<const float* const*>(e_loc), B, out2,
                                                        status, s));
  return DQ_OK;
}

dq_status mcmc_step_multi(dq_multi g, const void* const* params, void* const* r, void* const* logabs,
                          const int64_t* B, int32_t n_steps, double step_size, uint64_t seed, uint64_t step_counter,
                          uint64_t* step_counter_dev, int64_t* const* n_accepted, void* ws, size_t ws_bytes,
                          void* stream) {
  dq_status st = multi_args(g, B, {params, r, logabs});
  if (st != DQ_OK) return st;
  if (n_steps < 0 || !(step_size >= 0) || !isfinite(step_size)) return DQ_ERR_ARG;
  if (!entries_set(params, B, g->n) || !entries_set(r, B, g->n) || !entries_set(logabs, B, g->n)) return DQ_ERR_ARG;
  const cudaStream_t s = (cudaStream_t)stream;
  if (n_steps == 0) {
    for (int m = 0; m < g->n; ++m)
      if (n_accepted && n_accepted[m]) DQ_CU(cudaMemsetAsync(n_accepted[m], 0, sizeof(int64_t), s));
    return DQ_OK;
  }
  return run_mcmc_multi<float>(*g, reinterpret_cast<const float* const*>(params), reinterpret_cast<float* const*>(r),
                               reinterpret_cast<float* const*>(logabs), B, n_steps, step_size, seed,
                               step_counter_dev ? 0 : step_counter, step_counter_dev, n_accepted,
                               static_cast<unsigned char*>(ws), ws_bytes, s);
}

dq_status grad_logpsi_multi(dq_multi g, const void* const* params, const void* const* r, const int64_t* B,
                            const void* const* weights, void* const* grad_out, void* ws, size_t ws_bytes,
                            void* stream) {
  dq_status st = multi_args(g, B, {params, r, weights, grad_out});
  if (st != DQ_OK) return st;
  const MultiGradPlan plan = plan_grad_multi(*g, B, 4);
  if (!ws || ws_bytes < plan.total || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  auto* w = static_cast<unsigned char*>(ws);
  for (int m = 0; m < g->n; ++m) {
    st = grad_logpsi(g->h[m], params[m], r[m], B[m], weights[m], 0, grad_out[m], w + plan.off[m], plan.bytes[m],
                     stream);
    if (st != DQ_OK) return st;
  }
  return DQ_OK;
}

dq_status vmc_loss_weights_multi(dq_multi g, const void* const* e_loc, const int64_t* B, double clip_k,
                                 void* const* weights, double* const* stats, void* ws, size_t ws_bytes,
                                 void* stream) {
  dq_status st = multi_args(g, B, {e_loc, weights});
  if (st != DQ_OK) return st;
  if (!(clip_k > 0)) return DQ_ERR_ARG;
  for (int m = 0; m < g->n; ++m)
    if (B[m] < 1 || B[m] > 65536 || !e_loc[m] || !weights[m]) return DQ_ERR_ARG;
  size_t off[kMaxGroup];
  const size_t need = loss_scratch_multi(*g, B, off);
  if (!ws || ws_bytes < need || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  double* scratch[kMaxGroup];
  for (int m = 0; m < g->n; ++m) scratch[m] = reinterpret_cast<double*>(static_cast<unsigned char*>(ws) + off[m]);
  const cudaStream_t s = (cudaStream_t)stream;
  DQ_LAUNCH(*g->h[0], PK_LOSS_WEIGHTS,
            launch_loss_weights_group<float>(g->n, reinterpret_cast<const float* const*>(e_loc), B, clip_k,
                                             reinterpret_cast<float* const*>(weights), stats, scratch, s));
  return DQ_OK;
}

dq_status dq_set_msg_tile(dq_handle h, int32_t msg_ib) {
  if (!h || (msg_ib != 0 && msg_ib != 4 && msg_ib != 8)) return DQ_ERR_ARG;
  h->msg_ib = msg_ib;
  return DQ_OK;
}

dq_status dq_msg_tile(dq_handle h, int32_t* msg_ib) {
  if (!h || !msg_ib) return DQ_ERR_ARG;
  *msg_ib = h->msg_ib == 0 ? 8 : h->msg_ib;
  return DQ_OK;
}

dq_status dq_set_msg_kernel(dq_handle h, int32_t mode) {
  if (!h || mode < 0 || mode > 2) return DQ_ERR_ARG;
  if (mode == 2 && h->precision == DQ_FP64) return DQ_ERR_UNSUPPORTED;
  h->msg_kernel = mode;
  return DQ_OK;
}

dq_status dq_msg_kernel(dq_handle h, int32_t* mode) {
  if (!h || !mode) return DQ_ERR_ARG;
  const FwdDims d{1, h->N, h->n_up, h->n_dn, h->M, h->D, h->K, h->Q, 3 * h->N + 2};
  const bool tiled = h->msg_kernel == 2 || (h->msg_kernel == 0 && h->N > 16);
  *mode = tiled && messages_large_supported(*h, d) ? 2 : 1;
  return DQ_OK;
}

dq_status dq_set_layer_kernel(dq_handle h, int32_t mode) {
  if (!h || mode < 0 || mode > 2) return DQ_ERR_ARG;
  if (mode == 1 && !(use_tf32x3(*h) && layer_fused_supported(*h))) return DQ_ERR_UNSUPPORTED;
  h->layer_kernel = mode;
  return DQ_OK;
}

dq_status dq_layer_kernel(dq_handle h, int32_t* fused) {
  if (!h || !fused) return DQ_ERR_ARG;
  *fused = use_fused(*h, true) ? 1 : 0;
  return DQ_OK;
}

dq_status dq_set_det_warps(dq_handle h, int32_t warps) {
  if (!h || (warps != 2 && warps != 4)) return DQ_ERR_ARG;
  h->det_warps = warps;
  return DQ_OK;
}

dq_status dq_tile_set(dq_handle h, int64_t* max_chunk, int32_t* msg_ib, int32_t* layer_kernel, int32_t* det_warps) {
  if (!h || !max_chunk || !msg_ib || !layer_kernel || !det_warps) return DQ_ERR_ARG;
  *max_chunk = h->max_chunk;
  *msg_ib = h->msg_ib == 0 ? 8 : h->msg_ib;
  *layer_kernel = use_fused(*h, true) ? 1 : 2;
  *det_warps = h->det_warps;
  return DQ_OK;
}

namespace {
// Tile sets chosen by dq_autotune, per molecule size, ansatz shape, precision and walker count:
// a later handle of the same configuration takes the cached set instead of timing again.
struct TuneKey {
  int N, n_up, M, D, L, K, Q, precision, full_det, edge_update, el_init;
  int64_t B;
  bool operator<(const TuneKey& o) const {
    return std::tie(N, n_up, M, D, L, K, Q, precision, full_det, edge_update, el_init, B) <
           std::tie(o.N, o.n_up, o.M, o.D, o.L, o.K, o.Q, o.precision, o.full_det, o.edge_update, o.el_init, o.B);
  }
};
struct TuneVal {
  int64_t chunk;
  int ib, lk, dw;
  double ms;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;
TuneKey tune_key(const dq_handle_s& h, int64_t B) {
  return TuneKey{h.N, h.n_up, h.M, h.D, h.L, h.K, h.Q, (int)h.precision, h.full_det, h.edge_update, h.el_init, B};
}
}  // namespace

dq_status dq_autotune(dq_handle h, const void* params, const void* r, int64_t B, void* ws, size_t ws_bytes,
                      void* stream, double* best_ms) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (B < 1 || !params || !r || h->precision == DQ_FP64) return h->precision == DQ_FP64 ? DQ_ERR_UNSUPPORTED : DQ_ERR_ARG;
  if (!ws || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto it = g_tune_cache.find(tune_key(*h, B));
    if (it != g_tune_cache.end()) {
      h->max_chunk = it->second.chunk;
      h->msg_ib = it->second.ib;
      h->layer_kernel = it->second.lk;
      h->det_warps = it->second.dw;
      if (best_ms) *best_ms = it->second.ms;
      return DQ_OK;
    }
  }
  const cudaStream_t s = (cudaStream_t)stream;
  auto* w = static_cast<unsigned char*>(ws);
  // timing outputs after the largest candidate's forward workspace
  const int64_t keep_chunk = h->max_chunk;
  const int keep_ib = h->msg_ib;
  const int keep_lk = h->layer_kernel;
  // layer paths: the fused kernel where supported, and the separate kernels when the workspace
  // holds their message buffer
  const bool can_fuse = use_tf32x3(*h) && layer_fused_supported(*h);
  h->max_chunk = 4096;
  h->layer_kernel = can_fuse ? 1 : 2;
  const size_t fwd_f = align_up(plan_forward(*h, std::min<int64_t>(B, 4096), true, 4).total);
  h->layer_kernel = 2;
  const size_t fwd_s = align_up(plan_forward(*h, std::min<int64_t>(B, 4096), true, 4).total);
  h->max_chunk = keep_chunk;
  h->layer_kernel = keep_lk;
  const size_t b = (size_t)B;
  const size_t outs = 2 * align_up(b * 4) + align_up(b);
  const bool try_sep = !can_fuse || ws_bytes >= fwd_s + outs;
  const size_t fwd = try_sep ? std::max(fwd_f, fwd_s) : fwd_f;
  if (ws_bytes < fwd + outs) return DQ_ERR_WORKSPACE;
  float* la = reinterpret_cast<float*>(w + fwd);
  float* el = reinterpret_cast<float*>(w + fwd + align_up(b * 4));
  int8_t* sg = reinterpret_cast<int8_t*>(w + fwd + 2 * align_up(b * 4));
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return DQ_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return DQ_ERR_CUDA;
  }
  double best = -1;
  int64_t best_chunk = keep_chunk;
  const int keep_dw = h->det_warps;
  int best_ib = keep_ib, best_lk = keep_lk, best_dw = keep_dw;
  for (int lk : {1, 2}) {
    if ((lk == 1 && !can_fuse) || (lk == 2 && !try_sep)) continue;
    for (int64_t chunk : {(int64_t)4096, (int64_t)2048}) {
      // the message register tile matters only to the separate message kernel; the determinant
      // kernels' CTA size is tried with the largest chunk only
      for (int cand = 0; cand < 3; ++cand) {
        const int ib = cand == 1 ? 4 : 8, dw = cand == 2 ? 2 : 4;
        if ((lk == 1 && cand == 1) || (cand == 2 && chunk != 4096)) continue;
        h->layer_kernel = lk;
        h->max_chunk = chunk;
        h->msg_ib = ib;
        h->det_warps = dw;
        float ms = 0;
        for (int rep = 0; rep < 3 && st == DQ_OK; ++rep) {
          if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) st = DQ_ERR_CUDA;
          if (st == DQ_OK)
            st = run_forward<float>(*h, (const float*)params, (const float*)r, B, true, la, sg, el, w, fwd, s);
        }
        if (st != DQ_OK) break;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          st = DQ_ERR_CUDA;
          break;
        }
        if (best < 0 || ms / 2.0 < best) {
          best = ms / 2.0;
          best_chunk = chunk;
          best_ib = ib;
          best_lk = lk;
          best_dw = dw;
        }
      }
      if (st != DQ_OK) break;
    }
    if (st != DQ_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->max_chunk = st == DQ_OK ? best_chunk : keep_chunk;
  h->msg_ib = st == DQ_OK ? best_ib : keep_ib;
  h->layer_kernel = st == DQ_OK ? best_lk : keep_lk;
  h->det_warps = st == DQ_OK ? best_dw : keep_dw;
  if (st == DQ_OK) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[tune_key(*h, B)] = TuneVal{best_chunk, best_ib, best_lk, best_dw, best};
  }
  if (best_ms) *best_ms = best;
  return st;
}

dq_status dq_autotune_multi(dq_multi g, const void* const* params, const void* const* r, const int64_t* B, void* ws,
                            size_t ws_bytes, void* stream, double* best_ms) {
  dq_status st = multi_args(g, B, {params, r});
  if (st != DQ_OK) return st;
  if (!entries_set(params, B, g->n) || !entries_set(r, B, g->n)) return DQ_ERR_ARG;
  const size_t need = autotune_bytes(*g, B);
  if (!ws || ws_bytes < need || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  const cudaStream_t s = (cudaStream_t)stream;
  auto* w = static_cast<unsigned char*>(ws);
  // timing outputs at the end of the workspace
  size_t o = need;
  float *la[kMaxGroup], *el[kMaxGroup];
  int8_t* sg[kMaxGroup];
  for (int m = g->n - 1; m >= 0; --m) {
    const size_t b = (size_t)std::max<int64_t>(B[m], 1);
    o -= align_up(b);
    sg[m] = reinterpret_cast<int8_t*>(w + o);
    o -= align_up(b * 4);
    el[m] = reinterpret_cast<float*>(w + o);
    o -= align_up(b * 4);
    la[m] = reinterpret_cast<float*>(w + o);
  }
  const size_t fwd_bytes = o;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return DQ_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return DQ_ERR_CUDA;
  }
  const int keep_rounds = g->rounds;
  const int keep_ib = g->h[0]->msg_ib;
  double best = -1;
  int best_rounds = keep_rounds, best_ib = keep_ib;
  st = DQ_OK;
  for (int rounds = 1; rounds <= 4 && st == DQ_OK; ++rounds) {
    g->rounds = rounds;
    if (plan_forward_multi(*g, B, true, 4).total > fwd_bytes) continue;
    for (int ib : {8, 4}) {
      for (int m = 0; m < g->n; ++m) g->h[m]->msg_ib = ib;
      float ms = 0;
      for (int rep = 0; rep < 3 && st == DQ_OK; ++rep) {
        if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) st = DQ_ERR_CUDA;
        if (st == DQ_OK)
          st = run_forward_multi<float>(*g, reinterpret_cast<const float* const*>(params),
                                        reinterpret_cast<const float* const*>(r), B, true, la, sg, el, w, fwd_bytes,
                                        s);
      }
      if (st != DQ_OK) break;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        st = DQ_ERR_CUDA;
        break;
      }
      const double t = ms / 2.0;
      if (best < 0 || t < best) {
        best = t;
        best_rounds = rounds;
        best_ib = ib;
      }
    }
  }
  // the determinant kernels' CTA size, at the best rounds and message tile
  const int keep_dw = g->h[0]->det_warps;
  int best_dw = keep_dw;
  if (st == DQ_OK && best >= 0) {
    g->rounds = best_rounds;
    for (int dw : {4, 2}) {
      for (int m = 0; m < g->n; ++m) {
        g->h[m]->msg_ib = best_ib;
        g->h[m]->det_warps = dw;
      }
      float ms = 0;
      for (int rep = 0; rep < 3 && st == DQ_OK; ++rep) {
        if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) st = DQ_ERR_CUDA;
        if (st == DQ_OK)
          st = run_forward_multi<float>(*g, reinterpret_cast<const float* const*>(params),
                                        reinterpret_cast<const float* const*>(r), B, true, la, sg, el, w, fwd_bytes,
                                        s);
      }
      if (st != DQ_OK) break;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        st = DQ_ERR_CUDA;
        break;
      }
      if (dw == 2 && ms / 2.0 < best) {
        best = ms / 2.0;
        best_dw = 2;
      } else if (dw == 4) {
        best = std::min(best, ms / 2.0);  // the same candidate, timed again
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g->rounds = st == DQ_OK ? best_rounds : keep_rounds;
  for (int m = 0; m < g->n; ++m) {
    g->h[m]->msg_ib = st == DQ_OK ? best_ib : keep_ib;
    g->h[m]->det_warps = st == DQ_OK ? best_dw : keep_dw;
  }
  if (best_ms) *best_ms = best;
  return st;
}

dq_status dq_multi_tile_set(dq_multi g, int32_t* rounds, int32_t* msg_ib, int32_t* fused_layers,
                            int32_t* det_warps) {
  if (!g || !rounds || !msg_ib || !fused_layers || !det_warps) return DQ_ERR_ARG;
  *rounds = g->rounds;
  *msg_ib = g->h[0]->msg_ib == 0 ? 8 : g->h[0]->msg_ib;
  int f = 0;
  for (int m = 0; m < g->n; ++m) f += use_fused(*g->h[m], true) ? 1 : 0;
  *fused_layers = f;
  *det_warps = g->h[0]->det_warps;
  return DQ_OK;
}

dq_status dq_multi_tuning(dq_multi g, int32_t* rounds, int32_t* msg_ib) {
  if (!g || !rounds || !msg_ib) return DQ_ERR_ARG;
  *rounds = g->rounds;
  *msg_ib = g->h[0]->msg_ib == 0 ? 8 : g->h[0]->msg_ib;
  return DQ_OK;
}

}  // extern "C"
