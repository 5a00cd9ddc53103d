// A7: perturbation of Sec. III-A and the step matrices of the reduced
// leap-frog, all in FP64 on the GPU with small dense kernels written here:
// Cholesky (one CTA), triangular solves (a warp per right-hand side), GEMM,
// and a one-sided (Hestenes) Jacobi SVD run as one cooperative kernel with a
// round-robin pairing of columns.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mor_common.cuh"
#include "mor_internal.cuh"

namespace cg = cooperative_groups;

namespace fdtdmor {

// In-place Cholesky A = L L^T of the n x n row-major matrix (lower triangle
// returned, strict upper triangle zeroed).  info[0] = j+1 when the leading
// minor of order j+1 is not positive definite.
__global__ void __launch_bounds__(1024) chol_kernel(double *A, int n, int *info) {
  __shared__ double red[32];
  __shared__ double diag;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) info[0] = 0;
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int k = threadIdx.x; k < j; k += blockDim.x) s += A[j * n + k] * A[j * n + k];
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[w] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int q = 0; q < nw; ++q) t += red[q];
      const double d = A[j * n + j] - t;
      if (!(d > 0)) { info[0] = j + 1; diag = 0; }
      else { diag = sqrt(d); A[j * n + j] = diag; }
    }
    __syncthreads();
    if (diag == 0) return;
    for (int i = j + 1 + w; i < n; i += nw) {
      double d = 0;
      for (int k = lane; k < j; k += 32) d += A[i * n + k] * A[j * n + k];
      for (int o = 16; o; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
      if (lane == 0) A[i * n + j] = (A[i * n + j] - d) / diag;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < n * n; t += blockDim.x)
    if (t % n > t / n) A[t] = 0;
}

// Solve L X = B (trans = 0) or L^T X = B (trans = 1) in place; L n x n lower
// row-major, B n x ncols row-major.  One warp per column of B.
__global__ void trsm_kernel(const double *__restrict__ L, int n, double *B, int ncols, int trans) {
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= ncols) return;
  if (!trans) {
    for (int i = 0; i < n; ++i) {
      double d = 0;
      for (int k = lane; k < i; k += 32) d += L[i * n + k] * B[k * ncols + col];
      for (int o = 16; o; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
      if (lane == 0) B[i * ncols + col] = (B[i * ncols + col] - d) / L[i * n + i];
      __syncwarp();
    }
  } else {
    for (int i = n - 1; i >= 0; --i) {
      double d = 0;
      for (int k = i + 1 + lane; k < n; k += 32) d += L[k * n + i] * B[k * ncols + col];
      for (int o = 16; o; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
      if (lane == 0) B[i * ncols + col] = (B[i * ncols + col] - d) / L[i * n + i];
      __syncwarp();
    }
  }
}

// C = alpha op(A) op(B) + beta C; row-major; op(A) is M x K, op(B) K x N.
__global__ void gemm_f64_kernel(int M, int N, int K, double alpha, const double *__restrict__ A, int ta,
                                const double *__restrict__ Bm, int tb, double beta, double *C) {
  __shared__ double As[16][17], Bs[16][17];
  const int r = blockIdx.y * 16 + threadIdx.y, c = blockIdx.x * 16 + threadIdx.x;
  double acc = 0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    As[threadIdx.y][threadIdx.x] = (r < M && ka < K) ? (ta ? A[ka * M + r] : A[r * K + ka]) : 0.0;
    Bs[threadIdx.y][threadIdx.x] = (kb < K && c < N) ? (tb ? Bm[c * K + kb] : Bm[kb * N + c]) : 0.0;
    __syncthreads();
    for (int k = 0; k < 16; ++k) acc += As[threadIdx.y][k] * Bs[k][threadIdx.x];
    __syncthreads();
  }
  if (r < M && c < N) C[r * N + c] = alpha * acc + (beta == 0.0 ? 0.0 : beta * C[r * N + c]);
}

// Z = a X + b Y (elementwise), X or Y may alias Z.
__global__ void axpby_kernel(int n, double a, const double *X, double b, const double *Y, double *Z) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) Z[t] = a * X[t] + (Y ? b * Y[t] : 0.0);
}

__global__ void transpose_kernel(int rows, int cols, const double *__restrict__ A, double *__restrict__ At) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < rows * cols) At[(t % cols) * rows + t / cols] = A[t];
}

__global__ void eye_kernel(int n, double *A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n * n) A[t] = (t / n == t % n) ? 1.0 : 0.0;
}

template <typename T>
__global__ void convert_kernel(int n, const double *__restrict__ X, T *__restrict__ Y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) Y[t] = (T)X[t];
}

// One-sided Jacobi SVD of the m x n column-major matrix Mc: rotates column
// pairs until all are orthogonal (|a_p . a_q| <= tol ||a_p|| ||a_q||); the
// rotations accumulate in Wc (n x n column-major, identity on entry).  At the
// end Mc = U S and Mc_in = U S W^T.  flag[0] counts rotations of the current
// sweep, flag[1] receives the number of sweeps.
__global__ void __launch_bounds__(256) jacobi_svd_kernel(double *Mc, int m, int n, double *Wc, double tol,
                                                         int max_sweeps, unsigned *flag) {
  cg::grid_group grid = cg::this_grid();
  const int nn = n + (n & 1), npairs = nn / 2;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int round = 0; round < nn - 1; ++round) {
      for (int pr = gw; pr < npairs; pr += nwarps) {
        int a, b;
        if (pr == 0) { a = 0; b = (round % (nn - 1)) + 1; }
        else { a = ((round + pr) % (nn - 1)) + 1; b = ((round - pr + (nn - 1)) % (nn - 1)) + 1; }
        if (a >= n || b >= n) continue;
        double al = 0, be = 0, ga = 0;
        for (int r = lane; r < m; r += 32) {
          const double x = Mc[(size_t)a * m + r], y = Mc[(size_t)b * m + r];
          al += x * x; be += y * y; ga += x * y;
        }
        for (int o = 16; o; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        // (sqrt(al) sqrt(be): the product al * be may underflow for columns
        // in the null space)
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        // a rotation by an angle below rounding changes nothing: such a pair
        // counts as orthogonal, so noise-level columns cannot stall the sweeps
        if (al > 0 && be > 0 && fabs(ga) > tol * sqrt(al) * sqrt(be) && fabs(t) > 1e-15) {
          const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          for (int r = lane; r < m; r += 32) {
            const double x = Mc[(size_t)a * m + r], y = Mc[(size_t)b * m + r];
            Mc[(size_t)a * m + r] = c * x - s * y;
            Mc[(size_t)b * m + r] = s * x + c * y;
          }
          for (int r = lane; r < n; r += 32) {
            const double x = Wc[(size_t)a * n + r], y = Wc[(size_t)b * n + r];
            Wc[(size_t)a * n + r] = c * x - s * y;
            Wc[(size_t)b * n + r] = s * x + c * y;
          }
          if (lane == 0) atomicAdd(&flag[0], 1u);
        }
      }
      grid.sync();
    }
    const bool done = atomicAdd(&flag[0], 0u) == 0;
    grid.sync();
    if (grid.thread_rank() == 0) flag[0] = 0;
    grid.sync();
    if (done) break;
  }
  if (grid.thread_rank() == 0) flag[1] = (unsigned)sweep;
}

// sigma_c = ||Mc_c||, sigma'_c = sigma_c if sigma_c < lim else lim; Z_c = Mc_c sigma'/sigma.
__global__ void clip_kernel(double *Mc, int m, int n, double lim, double *sigma, int *nclip) {
  const int c = blockIdx.x;
  __shared__ double red[32];
  double s = 0;
  for (int r = threadIdx.x; r < m; r += blockDim.x) s += Mc[(size_t)c * m + r] * Mc[(size_t)c * m + r];
  for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    red[0] = sqrt(t);
  }
  __syncthreads();
  const double sg = red[0];
  const double sp = sg < lim ? sg : lim;
  if (threadIdx.x == 0) {
    sigma[c] = sg;
    if (!(sg < lim)) atomicAdd(nclip, 1);
  }
  const double f = sg > 0 ? sp / sg : 0.0;
  for (int r = threadIdx.x; r < m; r += blockDim.x) Mc[(size_t)c * m + r] *= f;
}

// ------------------------------------------------------------------ host
struct Dense {
  cudaStream_t s;
  fdtd_status gemm(int M, int N, int K, double alpha, const double *A, int ta, const double *B, int tb,
                   double beta, double *C) {
    if (M == 0 || N == 0) return FDTD_OK;
    dim3 blk(16, 16), grd((N + 15) / 16, (M + 15) / 16);
    gemm_f64_kernel<<<grd, blk, 0, s>>>(M, N, K, alpha, A, ta, B, tb, beta, C);
    return after_launch("gemm_f64_kernel");
  }
  fdtd_status chol(double *A, int n, int *info_dev, const char *what) {
    if (n == 0) return FDTD_OK;
    chol_kernel<<<1, 1024, 0, s>>>(A, n, info_dev);
    FDTD_CHECK(after_launch("chol_kernel"));
    int info = 0;
    FDTD_CHECK_CUDA(cudaMemcpyAsync(&info, info_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
    if (info) {
      set_error("%s is not positive definite (leading minor %d)", what, info);
      return FDTD_EUNSTABLE;
    }
    return FDTD_OK;
  }
  fdtd_status trsm(const double *L, int n, double *B, int ncols, int trans) {
    if (n == 0 || ncols == 0) return FDTD_OK;
    const int wpb = 8;
    trsm_kernel<<<(ncols + wpb - 1) / wpb, 32 * wpb, 0, s>>>(L, n, B, ncols, trans);
    return after_launch("trsm_kernel");
  }
  fdtd_status axpby(int n, double a, const double *X, double b, const double *Y, double *Z) {
    if (n == 0) return FDTD_OK;
    axpby_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, a, X, b, Y, Z);
    return after_launch("axpby_kernel");
  }
  fdtd_status transpose(int rows, int cols, const double *A, double *At) {
    if (rows * cols == 0) return FDTD_OK;
    transpose_kernel<<<(rows * cols + 255) / 256, 256, 0, s>>>(rows, cols, A, At);
    return after_launch("transpose_kernel");
  }
};

template <typename T>
static fdtd_status to_run_type(cudaStream_t s, const double *X, int n, DevBuf &dst) {
  FDTD_CHECK(dst.alloc(sizeof(T) * std::max(1, n), s));
  if (n) {
    convert_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(n, X, dst.as<T>());
    FDTD_CHECK(after_launch("convert_kernel"));
  }
  return FDTD_OK;
}

fdtd_status to_run_type_dispatch(mor_model *M, const double *X, int n, DevBuf &dst, cudaStream_t s);

__global__ void count_nonfinite_kernel(const double *__restrict__ x, int n, int *bad) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
    if (!isfinite(x[t])) atomicAdd(bad, 1);
}

// The projected matrices must be finite before they are factorised.
static fdtd_status check_finite(mor_model *M, cudaStream_t s) {
  DevBuf bad;
  FDTD_CHECK(bad.alloc(sizeof(int), s));
  FDTD_CHECK_CUDA(cudaMemsetAsync(bad.ptr, 0, sizeof(int), s));
  const DevBuf *mats[] = {&M->De, &M->Dse, &M->Dm, &M->Dsm, &M->K};
  const int sizes[] = {M->q1 * M->q1, M->q1 * M->q1, M->q2 * M->q2, M->q2 * M->q2, M->q1 * M->q2};
  for (int i = 0; i < 5; ++i) {
    if (sizes[i] == 0) continue;
    count_nonfinite_kernel<<<std::min(1024, (sizes[i] + 255) / 256), 256, 0, s>>>(mats[i]->as<double>(), sizes[i], bad.as<int>());
    FDTD_CHECK(after_launch("count_nonfinite_kernel"));
  }
  int h = 0;
  FDTD_CHECK_CUDA(cudaMemcpyAsync(&h, bad.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  bad.release(s);
  if (h) {
    set_error("the reduced matrices hold %d non-finite entries (a shifted solve diverged)", h);
    return FDTD_EUNSTABLE;
  }
  return FDTD_OK;
}

static fdtd_status perturb_and_prepare(mor_model *M, double dt, double gamma, int *n_clipped, cudaStream_t s) {
  const int q1 = M->q1, q2 = M->q2, m = M->m, p = M->p;
  Dense D{s};
  DevBuf wk, info, flag;
  const size_t nq = (size_t)std::max(q1, q2);
  // workspace: Le, Lm, X (q1 x q2), Xt/Mc (q2 x q1), W (q2 x q2), T1, T2 (q1 x q2), step RHS
  const size_t words = 2 * nq * nq + 8 * nq * nq + 4 * nq * std::max(1, m) + 16;
  FDTD_CHECK(wk.alloc(sizeof(double) * words, s));
  FDTD_CHECK(info.alloc(sizeof(int) * 4, s));
  FDTD_CHECK(flag.alloc(sizeof(unsigned) * 4, s));
  double *w = wk.as<double>();
  double *Le = w, *Lm = Le + nq * nq, *X = Lm + nq * nq, *Mc = X + nq * nq, *Wc = Mc + nq * nq;
  double *T1 = Wc + nq * nq, *T2 = T1 + nq * nq, *A2 = T2 + nq * nq, *B2 = A2 + nq * nq, *R2 = B2 + nq * nq;
  int *dinfo = info.as<int>();
  // ---- Sec. III-A step 1: factors and M = Le^{-1} K~ Lm^{-T}, SVD
  FDTD_CHECK_CUDA(cudaMemcpyAsync(Le, M->De.ptr, sizeof(double) * q1 * q1, cudaMemcpyDeviceToDevice, s));
  FDTD_CHECK_CUDA(cudaMemcpyAsync(Lm, M->Dm.ptr, sizeof(double) * q2 * q2, cudaMemcpyDeviceToDevice, s));
  FDTD_CHECK(check_finite(M, s));
  FDTD_CHECK(D.chol(Le, q1, dinfo, "D~eps"));
  FDTD_CHECK(D.chol(Lm, q2, dinfo, "D~mu"));
  int ncl = 0;
  if (q1 && q2) {
    FDTD_CHECK_CUDA(cudaMemcpyAsync(X, M->K.ptr, sizeof(double) * q1 * q2, cudaMemcpyDeviceToDevice, s));
    FDTD_CHECK(D.trsm(Le, q1, X, q2, 0));            // X = Le^{-1} K~        (q1 x q2)
    FDTD_CHECK(D.transpose(q1, q2, X, Mc));          // X^T                   (q2 x q1)
    FDTD_CHECK(D.trsm(Lm, q2, Mc, q1, 0));           // Lm^{-1} X^T = M^T: M column-major
    eye_kernel<<<(q2 * q2 + 255) / 256, 256, 0, s>>>(q2, Wc);
    FDTD_CHECK(after_launch("eye_kernel"));
    FDTD_CHECK_CUDA(cudaMemsetAsync(flag.ptr, 0, sizeof(unsigned) * 4, s));
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jacobi_svd_kernel, 256, 0);
    const int npairs = (q2 + 1) / 2;
    int blocks = std::max(1, std::min((npairs + 7) / 8, std::max(1, per) * nsm));
    // rotation threshold: a few ulps times sqrt(rows) (pairs closer to orthogonal
    // than rounding can certify are left alone)
    double tol = std::max(1e-12, 4.0 * 2.220446049250313e-16 * std::sqrt((double)q1));
    int maxsw = 80;
    unsigned *fl = flag.as<unsigned>();
    int mm = q1, nn = q2;
    void *args[] = {&Mc, &mm, &nn, &Wc, &tol, &maxsw, &fl};
    FDTD_CHECK_CUDA(cudaLaunchCooperativeKernel((void *)jacobi_svd_kernel, dim3(blocks), dim3(256), args, 0, s));
    FDTD_CHECK(after_launch("jacobi_svd_kernel"));
    // ---- step 2: clip
    const double lim = gamma * 2.0 / dt;
    FDTD_CHECK_CUDA(cudaMemsetAsync(dinfo + 1, 0, sizeof(int), s));
    clip_kernel<<<q2, 128, 0, s>>>(Mc, q1, q2, lim, M->sigma.as<double>(), dinfo + 1);
    FDTD_CHECK(after_launch("clip_kernel"));
    // ---- step 3: K~' = Le U S' W^T Lm^T  (Mc now holds U S' column-major)
    FDTD_CHECK(D.gemm(q1, q2, q2, 1.0, Mc, 1, Wc, 0, 0.0, T1));   // (U S') W^T
    FDTD_CHECK(D.gemm(q1, q2, q1, 1.0, Le, 0, T1, 0, 0.0, T2));   // Le (.)
    FDTD_CHECK(D.gemm(q1, q2, q2, 1.0, T2, 0, Lm, 1, 0.0, M->Kp.as<double>()));  // (.) Lm^T
    FDTD_CHECK_CUDA(cudaMemcpyAsync(&ncl, dinfo + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    unsigned fh[2];
    FDTD_CHECK_CUDA(cudaMemcpyAsync(fh, fl, sizeof(fh), cudaMemcpyDeviceToHost, s));
    FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
    if ((int)fh[1] >= maxsw) {
      set_error("Jacobi SVD did not converge in %d sweeps", maxsw);
      return FDTD_ENOCONV;
    }
  }
  // singular values of the rectangular case beyond min(q1, q2) are zero: count
  // only the clipped ones (clip_kernel counted over q2 columns)
  M->n_clipped = ncl;
  if (n_clipped) *n_clipped = ncl;
  // ---- step matrices of the reduced leap-frog at dt
  // Ae = D~e/dt + D~se/2 = Le2 Le2^T; Pe = Ae^{-1}(D~e/dt - D~se/2), Qe = Ae^{-1} K~', be = Ae^{-1} B~_E
  FDTD_CHECK(D.axpby(q1 * q1, 1.0 / dt, M->De.as<double>(), 0.5, M->Dse.as<double>(), A2));
  FDTD_CHECK(D.chol(A2, q1, dinfo, "D~eps/dt + D~se/2"));
  auto solve_sym = [&](const double *L, int n, double *Bm, int nc) -> fdtd_status {
    FDTD_CHECK(D.trsm(L, n, Bm, nc, 0));
    return D.trsm(L, n, Bm, nc, 1);
  };
  FDTD_CHECK(D.axpby(q1 * q1, 1.0 / dt, M->De.as<double>(), -0.5, M->Dse.as<double>(), B2));
  FDTD_CHECK(solve_sym(A2, q1, B2, q1));
  FDTD_CHECK(to_run_type_dispatch(M, B2, q1 * q1, M->Pe, s));
  FDTD_CHECK_CUDA(cudaMemcpyAsync(R2, M->Kp.ptr, sizeof(double) * q1 * q2, cudaMemcpyDeviceToDevice, s));
  FDTD_CHECK(solve_sym(A2, q1, R2, q2));
  FDTD_CHECK(to_run_type_dispatch(M, R2, q1 * q2, M->Qe, s));
  FDTD_CHECK_CUDA(cudaMemcpyAsync(R2, M->BE.ptr, sizeof(double) * q1 * m, cudaMemcpyDeviceToDevice, s));
  FDTD_CHECK(solve_sym(A2, q1, R2, m));
  FDTD_CHECK(to_run_type_dispatch(M, R2, q1 * m, M->be, s));
  // Ah = D~m/dt + D~sm/2; Ph = Ah^{-1}(D~m/dt - D~sm/2), Qh = Ah^{-1} K~'^T, bh = Ah^{-1} B~_H
  FDTD_CHECK(D.axpby(q2 * q2, 1.0 / dt, M->Dm.as<double>(), 0.5, M->Dsm.as<double>(), A2));
  FDTD_CHECK(D.chol(A2, q2, dinfo, "D~mu/dt + D~sm/2"));
  FDTD_CHECK(D.axpby(q2 * q2, 1.0 / dt, M->Dm.as<double>(), -0.5, M->Dsm.as<double>(), B2));
  FDTD_CHECK(solve_sym(A2, q2, B2, q2));
  FDTD_CHECK(to_run_type_dispatch(M, B2, q2 * q2, M->Ph, s));
  FDTD_CHECK(D.transpose(q1, q2, M->Kp.as<double>(), R2));
  FDTD_CHECK(solve_sym(A2, q2, R2, q1));
  FDTD_CHECK(to_run_type_dispatch(M, R2, q2 * q1, M->Qh, s));
  FDTD_CHECK_CUDA(cudaMemcpyAsync(R2, M->BH.ptr, sizeof(double) * q2 * m, cudaMemcpyDeviceToDevice, s));
  FDTD_CHECK(solve_sym(A2, q2, R2, m));
  FDTD_CHECK(to_run_type_dispatch(M, R2, q2 * m, M->bh, s));
  FDTD_CHECK(to_run_type_dispatch(M, M->CE.as<double>(), p * q1, M->Cr, s));
  FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  M->dt = dt;
  M->perturbed = true;
  wk.release(s);
  info.release(s);
  flag.release(s);
  return FDTD_OK;
}

fdtd_status to_run_type_dispatch(mor_model *M, const double *X, int n, DevBuf &dst, cudaStream_t s) {
  return M->prec == FDTD_F64 ? to_run_type<double>(s, X, n, dst) : to_run_type<float>(s, X, n, dst);
}

}  // namespace fdtdmor

using namespace fdtdmor;

extern "C" {

fdtd_status mor_perturb(mor_model *M, double dt, double gamma, int *n_clipped, fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(M, "mor_perturb: NULL model");
  FDTD_REQUIRE(dt > 0 && gamma > 0 && gamma <= 1, "mor_perturb: need dt > 0 and 0 < gamma <= 1");
  return perturb_and_prepare(M, dt, gamma, n_clipped, (cudaStream_t)stream);
}

}  // extern "C"
