// Limits and handle internals shared by the reduction translation units.
#pragma once
#include "mor_common.cuh"

namespace fdtdmor {
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
  int64_t n3 = 0;
  int elem = 4;
  fdtd_prec prec = FDTD_F32;
  fdtdmor::DevBuf V1, V2;
  int max_iters = 0;
  double max_resid = 0;
  cudaStream_t stream = nullptr;
};
