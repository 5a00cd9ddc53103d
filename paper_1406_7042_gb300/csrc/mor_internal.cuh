// Limits and handle internals shared by the reduction translation units.
#pragma once
#include "mor_common.cuh"

namespace fdtdmor {

// Gram products on the CUDA cores (mor_project.cu): G = A^T B, columns of
// length n (stride n), FP64 out.
fdtd_status gram_native(cudaStream_t s, int64_t n, const float *A, int M, const float *B, int N, double *out);
fdtd_status gram_native(cudaStream_t s, int64_t n, const double *A, int M, const double *B, int N, double *out);
// dL/d eps per edge (FP64, 3 nc) -> per cell and per material (adjoint.cu).
fdtd_status edges_to_cells(fdtd_grid *g, const double *gedge, double *gcell, double *gmat, cudaStream_t s);

// Tensor-core Gram products (gram_tc.cu): G = A^T diag(w) B, FP64 out.
fdtd_status gram_pack(cudaStream_t s, bool bf16, int64_t n, int64_t n_pad, const float *src, int64_t ld, int ncols,
                      const float *w, void *dst);
fdtd_status gram_tensor_kmajor(cudaStream_t s, bool bf16, int64_t n, const void *A, int64_t lda, int M,
                               const void *B, int64_t ldb, int N, double *out, unsigned *err, DevBuf &part,
                               bool accumulate = false, int64_t max_rows = 0);
// Split-precision (three-pass) tensor-core Gram product: FP32-level accuracy.
fdtd_status gram_tensor_split(cudaStream_t s, bool bf16, int64_t n, const float *A, int64_t lda, int M, const float *B,
                              int64_t ldb, int N, const float *w, double *out, unsigned *err);
fdtd_status gram_tensor(cudaStream_t s, bool bf16, int64_t n, const float *A, int64_t lda, int M, const float *B,
                        int64_t ldb, int N, const float *w, double *out, unsigned *err);
constexpr int kMaxRhs = 16;   // expansion points x ports solved together
constexpr int kMaxDots = 64;  // columns per multi-dot pass
constexpr int kMaxRestarts = 8;  // true-residual restarts of a shifted solve

// Reduced model state (matrices in FP64 on the device, step matrices and the
// reduced state in the grid's type).
struct ModelState {
  int q1 = 0, q2 = 0, m = 0, p = 0;
  fdtd_prec prec = FDTD_F32;
  int elem = 4;
  DevBuf De, Dse, Dm, Dsm, K, Kp, BE, BH, CE, sigma;   // FP64
  DevBuf Pe, Qe, be, Ph, Qh, bh, Cr;                    // run type
  DevBuf state;                                         // e (q1) then h (q2), run type
  double dt = 0;
  int n_clipped = -1;
  bool perturbed = false;
  cudaStream_t stream = nullptr;
};
}  // namespace fdtdmor

struct mor_model : fdtdmor::ModelState {};

struct mor_basis {
  int q1 = 0, q2 = 0;
  int orth = 0;                 // mor_orth of the Gram-Schmidt products (used again by mor_project)
  int64_t n3 = 0;
  int elem = 4;
  fdtd_prec prec = FDTD_F32;
  fdtdmor::DevBuf V1, V2;
  int max_iters = 0;
  double max_resid = 0;
  cudaStream_t stream = nullptr;
};
