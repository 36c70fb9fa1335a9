// Launchers of the reverse pass (backward.cu).
#pragma once

#include "common.cuh"

namespace dq {

template <class T>
cudaError_t launch_bwd_combine(const dq_handle_s& h, int64_t Bc, const double* det, const T* jh, const T* params,
                               const T* weights, T* beta, T* cbar, T* jhbar, T* gt, cudaStream_t s);
template <class T>
cudaError_t launch_bwd_det(const dq_handle_s& h, int64_t Bc, const T* phi, const T* geo, const T* params, const T* beta,
                           T* phibar, T* envbar, cudaStream_t s);
// Y[r][n] (+)= sum_k X[r][k] W[k][n], W row-major [K][n_out]; any sizes.
template <class T>
cudaError_t gemm_nn(const T* X, RowMap mx, const T* W, T* Y, RowMap my, int64_t rows, int n_out, int K,
                    bool accumulate, cudaStream_t s);
// Parameter gradient block from rows: per walker (mode 1) writes G[b][off + o*ld + a],
// summed over walkers (mode 0) adds to G[off + o*ld + a]; Y == nullptr means ones.
// tc_status != nullptr allows the tensor-core row reduction (FP32, summed mode, large blocks);
// it receives DQ_FLAG_TIMEOUT if a bounded wait inside that kernel gave up.  done: nullptr or
// kColsumReduceCounters zeroed counters (left zeroed) with which summed-mode column sums add their
// splits in their last CTA instead of a second launch.
constexpr int kColsumReduceCounters = 64;
// boff >= 0: also the bias-type gradient G[boff + o] = sum_r X[r][o] where the tensor-core path runs
// (its column sums ride on the same pass over X); *bias_done tells whether it was formed.
template <class T>
cudaError_t param_reduce(const T* X, RowMap mx, const T* Y, RowMap my, int rpw, int64_t nw, int n_o, int n_a, T* G,
                         int64_t P, int64_t off, int ld, int mode, T* part, int64_t part_elems, cudaStream_t s,
                         unsigned int* tc_status = nullptr, unsigned int* done = nullptr, int64_t boff = -1,
                         bool* bias_done = nullptr);
template <class T>
cudaError_t launch_tanh_bwd(const T* g, const T* u, int64_t n, bool is_pre, T* out, cudaStream_t s);
template <class T>
cudaError_t launch_add_rows(T* fbar, const T* sbar, int64_t Bc, int N, int D, cudaStream_t s);
// Reverse of layer l's edge-embedding update: abar = ebar (1 - tanh^2(U f + c)) with f = fprev, then
// ebar <- ebar + U^T abar in place (rows [Bc * E][Q]).
template <class T>
cudaError_t launch_edge_update_bwd(const dq_handle_s& h, int64_t Bc, int l, const T* params, const T* fprev, T* ebar,
                                   T* abar, cudaStream_t s);
template <class T>
cudaError_t launch_fill_spin_rows(T* F0, const T* E_spin, int64_t Bc, int N, int n_up, int D, cudaStream_t s);
template <class T>
cudaError_t launch_msg_bwd(const dq_handle_s& h, int64_t Bc, const T* mbar, const T* Z, const T* z0, const T* ew,
                           const T* Y, bool z_const, T* zbar, T* wbar, T* ybar, cudaStream_t s);

}  // namespace dq
