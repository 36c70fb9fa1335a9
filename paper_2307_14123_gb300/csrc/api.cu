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
#include <new>
#include <vector>

#include "common.cuh"

namespace dq {

ParamOffsets make_offsets(int D, int L, int K, int Q, int M, int n_up, int n_dn) {
  ParamOffsets o{};
  int64_t p = 0;
  o.E_spin = p;
  p += 2 * (int64_t)D;
  for (int l = 0; l < L; ++l) {
    auto& y = o.layer[l];
    y.W_h = p;
    p += (int64_t)D * D;
    for (int t = 0; t < 3; ++t) {
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
  const int ns[2] = {n_up, n_dn};
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
                                          "gemm_jastrow", "combine", "layer0_node"};
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
  size_t geo, rbf, eh, ew, F, Z, msg, phi, det, js, jh, z0, total;
};

FwdPlan plan_forward(const dq_handle_s& h, int64_t Bc, bool jets, size_t elem) {
  const int64_t E = h.edges.n_all, N = h.N, D = h.D, K = h.K;
  const int64_t ej = jets ? 3 : 1, C = jets ? 3 * N + 2 : 1;
  const int64_t nmax = std::max(h.n_up, h.n_dn);
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
  p.F = take(Bc * N * C * D * elem);
  p.Z = take(Bc * N * C * D * elem);
  p.msg = take(Bc * N * C * 3 * D * elem);
  p.phi = take(Bc * N * C * K * nmax * elem);
  p.det = take(Bc * 2 * K * (3 * N + 3) * sizeof(double));
  p.js = take(Bc * C * D * elem);
  p.jh = take(Bc * C * D * elem);
  p.z0 = take(2 * D * elem);
  p.total = o;
  return p;
}

struct McmcPlan {
  size_t r_prop, la_prop, sign_prop, fwd, total;
};

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
                      int8_t* sign, T* e_loc, unsigned char* ws, size_t ws_bytes, cudaStream_t s) {
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

  const int N = h.N, D = h.D, K = h.K;
  const int C = jets ? 3 * N + 2 : 1;
  const int ej = jets ? 3 : 1;
  const int E = h.edges.n_all;
  const int nmax = std::max(h.n_up, h.n_dn);
  const int Wo = K * nmax;
  const int kb = jets ? 0 : kValueOffset;
  DQ_LAUNCH(h, kb + PK_LAYER0, launch_layer0_node<T>(h, FwdDims{Bmax, N, h.n_up, h.n_dn, h.M, D, K, h.Q, C}, params, bf, s));
  for (int64_t b0 = 0; b0 < B; b0 += Bmax) {
    const int64_t nb = std::min<int64_t>(Bmax, B - b0);
    const FwdDims d{nb, N, h.n_up, h.n_dn, h.M, D, K, h.Q, C};
    DQ_LAUNCH(h, kb + PK_GEOMETRY, launch_geometry<T>(h, d, r + b0 * N * 3, bf, s));
    for (int l = 0; l < h.L; ++l) {
      const auto& y = h.off.layer[l];
      DQ_LAUNCH(h, kb + PK_EDGE_HIDDEN, launch_edge_hidden<T>(h, d, params, l, bf, s));
      const int e0[3] = {0, h.edges.n_par, h.edges.n_ee};
      const int ng[3] = {h.edges.n_par, h.edges.n_anti, h.edges.n_en};
      for (int t = 0; t < 3; ++t) {
        if (ng[t] == 0) continue;
        const RowMap m{(int64_t)ng[t] * ej, (int64_t)E * ej * D, D};
        DQ_LAUNCH(h, kb + PK_GEMM_EDGE, gemm_nt<T>(bf.eh + (int64_t)e0[t] * ej * D, m, params + y.W2[t], params + y.b2[t], ej,
                         bf.ew + (int64_t)e0[t] * ej * D, m, nb * ng[t] * ej, D, D, false, s));
      }
      const RowMap node{(int64_t)N * C, (int64_t)N * C * D, D};
      if (l == 0) {
        DQ_LAUNCH(h, kb + PK_MESSAGES, launch_messages<T>(h, d, params, l, true, bf, s));
      } else {
        DQ_LAUNCH(h, kb + PK_GEMM_NODE, gemm_nt<T>(bf.F, node, params + y.W_h, nullptr, 1, bf.Z, node, nb * N * C, D, D, false, s));
        DQ_LAUNCH(h, kb + PK_MESSAGES, launch_messages<T>(h, d, params, l, false, bf, s));
      }
      const RowMap mrow{(int64_t)N * C, (int64_t)N * C * 3 * D, 3 * D};
      DQ_LAUNCH(h, kb + PK_GEMM_UPDATE, gemm_nt<T>(bf.msg, mrow, params + y.W_g, params + y.b_g, C, bf.Z, node, nb * N * C, D, 3 * D, false, s));
      DQ_LAUNCH(h, kb + PK_UPDATE, launch_update<T>(h, d, params, l == 0, bf, s));
    }
    const int ns[2] = {h.n_up, h.n_dn}, i0[2] = {0, h.n_up};
    for (int sg = 0; sg < 2; ++sg) {
      if (ns[sg] == 0) continue;
      const RowMap mx{(int64_t)ns[sg] * C, (int64_t)N * C * D, D};
      const RowMap my{(int64_t)ns[sg] * C, (int64_t)N * C * Wo, Wo};
      DQ_LAUNCH(h, kb + PK_GEMM_ORBITAL, gemm_nt<T>(bf.F + (int64_t)i0[sg] * C * D, mx, params + h.off.W_o[sg], params + h.off.b_o[sg], C,
                       bf.phi + (int64_t)i0[sg] * C * Wo, my, nb * ns[sg] * C, K * ns[sg], D, false, s));
    }
    DQ_LAUNCH(h, kb + PK_ORBITAL_DET, launch_orbital_det<T>(h, d, params, bf, s));
    if (h.use_jastrow) {
      DQ_LAUNCH(h, kb + PK_JASTROW_SUM, launch_jastrow_sum<T>(h, d, bf, s));
      const RowMap mj{(int64_t)C, (int64_t)C * D, D};
      DQ_LAUNCH(h, kb + PK_GEMM_JASTROW, gemm_nt<T>(bf.js, mj, params + h.off.W_J1, params + h.off.b_J1, C, bf.jh, mj, nb * C, D, D, false, s));
    }
    DQ_LAUNCH(h, kb + PK_COMBINE, launch_combine<T>(h, d, params, bf, logabs + b0, sign + b0, e_loc ? e_loc + b0 : nullptr, s));
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
                   uint64_t seed, uint64_t t0, int64_t* n_acc, unsigned char* ws, size_t ws_bytes, cudaStream_t s) {
  const McmcPlan plan = plan_mcmc(*h, B, sizeof(T));
  if (ws == nullptr || ws_bytes < plan.total || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  T* r_prop = reinterpret_cast<T*>(ws + plan.r_prop);
  T* la_prop = reinterpret_cast<T*>(ws + plan.la_prop);
  int8_t* sg_prop = reinterpret_cast<int8_t*>(ws + plan.sign_prop);
  if (n_acc) DQ_CU(cudaMemsetAsync(n_acc, 0, sizeof(int64_t), s));
  for (int32_t k = 0; k < n_steps; ++k) {
    const uint64_t t = t0 + (uint64_t)k;
    DQ_LAUNCH(*h, PK_PROPOSE, launch_propose<T>(*h, B, r, r_prop, step, seed, t, s));
    dq_status st = run_forward<T>(*h, params, r_prop, B, false, la_prop, sg_prop, nullptr, ws + plan.fwd,
                                  ws_bytes - plan.fwd, s);
    if (st != DQ_OK) return st;
    DQ_LAUNCH(*h, PK_ACCEPT, launch_accept<T>(*h, B, r, logabs, r_prop, la_prop, sg_prop, seed, t,
                           reinterpret_cast<unsigned long long*>(n_acc), s));
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
  if (precision != DQ_FP64 && precision != DQ_FP32) return precision == DQ_BF16_MIXED ? DQ_ERR_UNSUPPORTED : DQ_ERR_ARG;
  if (!sys->Z || !sys->R) return DQ_ERR_ARG;
  const int M = sys->n_nuc, n_up = sys->n_up, n_dn = sys->n_down, N = n_up + n_dn;
  if (M < 1 || M > kMaxNuc || n_up < 1 || n_dn < 0 || N > kMaxElec || n_up > kMaxSpin || n_dn > kMaxSpin)
    return DQ_ERR_SHAPE;
  if (cfg->width < 32 || cfg->width % 32 || cfg->width > 512 || cfg->n_layers < 1 || cfg->n_layers > kMaxLayers ||
      cfg->n_det < 1 || cfg->n_det > 128 || cfg->n_rbf < 8 || cfg->n_rbf % 8 || cfg->n_rbf > 64 ||
      !(cfg->rbf_cutoff > 0) || !(cfg->cusp_alpha > 0))
    return DQ_ERR_SHAPE;
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
  h->off = make_offsets(h->D, h->L, h->K, h->Q, M, n_up, n_dn);
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
            cudaMalloc(&h->d_status, sizeof(unsigned int)) == cudaSuccess;
  ok = ok && cudaMemcpy(h->d_R, sys->R, 3 * M * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(h->d_Rf, Rf.data(), 3 * M * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(h->d_Z, sys->Z, M * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(h->d_pair_of, pof.data(), N * N * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(h->d_pair_ij, pij.data(), pij.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(h->d_status, 0, sizeof(unsigned int)) == cudaSuccess;
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
    case DQ_OP_GRAD: *bytes = 0; return DQ_ERR_UNSUPPORTED;
    case DQ_OP_LOSS_WEIGHTS: *bytes = loss_scratch_bytes(std::max<int64_t>(B, 1)); return DQ_OK;
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


dq_status mcmc_step(dq_handle h, const void* params, void* r, void* logabs, int64_t B, int32_t n_steps,
                    double step_size, uint64_t seed, uint64_t step_counter, int64_t* n_accepted, void* ws,
                    size_t ws_bytes, void* stream) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (B < 0 || n_steps < 0 || !(step_size >= 0) || !isfinite(step_size)) return DQ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (B == 0 || n_steps == 0) {
    if (n_accepted && cudaMemsetAsync(n_accepted, 0, sizeof(int64_t), s) != cudaSuccess) return DQ_ERR_CUDA;
    return DQ_OK;
  }
  if (!params || !r || !logabs) return DQ_ERR_ARG;
  auto* w = static_cast<unsigned char*>(ws);
  if (h->precision == DQ_FP64)
    return run_mcmc<double>(h, (const double*)params, (double*)r, (double*)logabs, B, n_steps, step_size, seed,
                            step_counter, n_accepted, w, ws_bytes, s);
  return run_mcmc<float>(h, (const float*)params, (float*)r, (float*)logabs, B, n_steps, step_size, seed,
                         step_counter, n_accepted, w, ws_bytes, s);
}

dq_status grad_logpsi(dq_handle h, const void* params, const void* r, int64_t B, const void* weights, int32_t mode,
                      void* grad_out, void* ws, size_t ws_bytes, void* stream) {
  (void)params; (void)r; (void)B; (void)weights; (void)mode; (void)grad_out; (void)ws; (void)ws_bytes; (void)stream;
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  return DQ_ERR_UNSUPPORTED;
}

dq_status vmc_loss_weights(dq_handle h, const void* e_loc, int64_t B, double clip_k, void* weights, double* stats,
                           void* ws, size_t ws_bytes, void* stream) {
  dq_status st = check_handle(h);
  if (st != DQ_OK) return st;
  if (B < 1 || B > 65536 || !e_loc || !weights || !(clip_k > 0)) return DQ_ERR_ARG;
  if (!ws || ws_bytes < loss_scratch_bytes(B) || !aligned(ws, kAlign)) return DQ_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (h->precision == DQ_FP64)
    DQ_LAUNCH(*h, PK_LOSS_WEIGHTS, launch_loss_weights<double>((const double*)e_loc, B, clip_k, (double*)weights, stats, (double*)ws, s));
  else
    DQ_LAUNCH(*h, PK_LOSS_WEIGHTS, launch_loss_weights<float>((const float*)e_loc, B, clip_k, (float*)weights, stats, (double*)ws, s));
  return DQ_OK;
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

int32_t dq_profile_kind_count(void) { return PK_COUNT; }

}  // extern "C"
