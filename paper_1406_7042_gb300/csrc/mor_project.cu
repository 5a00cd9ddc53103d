// A6: structure-preserving projection, Eq. (R_and_Freduced):
//   D~eps = V1^T D_eps V1, D~se = V1^T D_se V1, D~mu = V2^T D_mu V2,
//   D~sm = V2^T D_sm V2, K~ = V1^T K V2, B~ = V^T B, C~ = C V.
// The diagonal D matrices carry the edge volumes of Eq. (matrix) (D_eps =
// eps_e A~_e L_e, ...), K = -V_e curl_H, and B = -w V_e at the source edges.
// Products are tall-skinny Gram products V_a^T diag(w) V_b over the 3 nc rows:
// each CTA accumulates a 32 x 32 output tile over a slice of rows in the
// field type and adds the slice into FP64 partial sums, which a second
// kernel adds over slices.
#include <algorithm>
#include <cstdlib>
#include <string>
#include <utility>
#include <vector>

#include "grid_internal.cuh"
#include "mor_common.cuh"
#include "mor_internal.cuh"

namespace fdtdmor {

// Per-edge diagonal weights: 0: D_eps, 1: D_se (E edges), 2: D_mu, 3: D_sm (H edges).
template <typename T>
__global__ void diag_weights_kernel(Geo<T> g, const T *__restrict__ ep, T *__restrict__ out) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = g.nc;
  if (n >= nc) return;
  const int i = (int)(n % g.nx), j = (int)((n / g.nx) % g.ny), k = (int)(n / ((int64_t)g.nx * g.ny));
  const int idx[3] = {i, j, k};
  for (int c = 0; c < 3; ++c) {
    const int64_t e = c * nc + n;
    // E edge along axis c: length d_c, dual face of the other two dual spacings
    const T eps = ep[EP_EPS * 3 * nc + e];
    T ve = 0;
    if (eps != T(0)) {
      const int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
      ve = T(1) / (g.rd(c, idx[c]) * g.rdd(a1, idx[a1]) * g.rdd(a2, idx[a2]));
    }
    out[0 * 3 * nc + e] = eps * ve;
    out[1 * 3 * nc + e] = ep[EP_SIG * 3 * nc + e] * ve;
    // H edge along axis c: dual length, primal face of the other two spacings
    const T mu = ep[EP_MU * 3 * nc + e];
    T vh = 0;
    if (mu != T(0)) {
      const int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
      vh = T(1) / (g.rdd(c, idx[c]) * g.rd(a1, idx[a1]) * g.rd(a2, idx[a2]));
    }
    out[2 * 3 * nc + e] = mu * vh;
    out[3 * 3 * nc + e] = ep[EP_SGM * 3 * nc + e] * vh;
  }
}

// W[c] = K V2[c] = -V_e curl_H(V2[c]) on live E edges.
template <typename T>
__global__ void kv_kernel(Geo<T> g, const T *__restrict__ ep, const T *__restrict__ V2, T *__restrict__ W) {
  const int col = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = g.nc;
  if (n >= nc) return;
  const int i = (int)(n % g.nx), j = (int)((n / g.nx) % g.ny), k = (int)(n / ((int64_t)g.nx * g.ny));
  const T *v = V2 + (size_t)col * 3 * nc;
  auto ld = [&](int64_t idx) { return v[idx]; };
  const int idx[3] = {i, j, k};
  for (int c = 0; c < 3; ++c) {
    const int64_t e = c * nc + n;
    T out = 0;
    if (ep[EP_EPS * 3 * nc + e] != T(0)) {
      const int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
      const T ve = T(1) / (g.rd(c, idx[c]) * g.rdd(a1, idx[a1]) * g.rdd(a2, idx[a2]));
      out = -ve * curl_h_at<T, T>(g, ld, c, i, j, k);
    }
    W[(size_t)col * 3 * nc + e] = out;
  }
}

constexpr int GT = 32;   // output tile
constexpr int GK = 32;   // rows per smem stage

// partial[s][a][b] = sum over rows of slice s of A[a][r] w[r] B[b][r]
template <typename T>
__global__ void __launch_bounds__(256) gram_kernel(int64_t nrows, const T *__restrict__ A, int qa,
                                                   const T *__restrict__ Bm, int qb, const T *__restrict__ w,
                                                   int64_t slice, double *__restrict__ partial) {
  __shared__ T As[GK][GT + 1];
  __shared__ T Bs[GK][GT + 1];
  const int a0 = blockIdx.x * GT, b0 = blockIdx.y * GT;
  const int64_t r_beg = (int64_t)blockIdx.z * slice, r_end = min(nrows, r_beg + slice);
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // ty: 0..7 -> 4 rows of a each
  double acc64[4] = {0, 0, 0, 0};
  T acc[4] = {0, 0, 0, 0};
  int since = 0;
  for (int64_t r0 = r_beg; r0 < r_end; r0 += GK) {
    // load GK rows x 32 columns of A and B (transposed into [row][col])
    for (int t = threadIdx.x; t < GK * GT; t += 256) {
      const int rr = t % GK, cc = t / GK;
      const int64_t r = r0 + rr;
      T av = 0, bv = 0;
      if (r < r_end) {
        if (a0 + cc < qa) av = A[(size_t)(a0 + cc) * nrows + r];
        if (b0 + cc < qb) {
          bv = Bm[(size_t)(b0 + cc) * nrows + r];
          if (w) bv *= w[r];
        }
      }
      As[rr][cc] = av;
      Bs[rr][cc] = bv;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < GK; ++rr) {
      const T bv = Bs[rr][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += As[rr][ty * 4 + q] * bv;
    }
    __syncthreads();
    if (++since == 8) {  // fold the field-type partial into FP64 every 256 rows
      for (int q = 0; q < 4; ++q) { acc64[q] += (double)acc[q]; acc[q] = 0; }
      since = 0;
    }
  }
  for (int q = 0; q < 4; ++q) acc64[q] += (double)acc[q];
  for (int q = 0; q < 4; ++q) {
    const int a = a0 + ty * 4 + q, b = b0 + tx;
    if (a < qa && b < qb) partial[((size_t)blockIdx.z * qa + a) * qb + b] = acc64[q];
  }
}

__global__ void sum_slices_kernel(int nslice, int n, const double *__restrict__ partial, double *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double a = 0;
  for (int s = 0; s < nslice; ++s) a += partial[(size_t)s * n + t];
  out[t] = a;
}

// B~[a][p] += sum over port edges of V1[a][e] * val[e] (val = -w V_e for
// sources, w for probes); output row-major [a][p] (or [p][a] with transpose).
struct PortEdge {
  int64_t e;   // index into the 3 nc E vector
  int port;
  int by_volume;  // 1: value -w V_e (a column of B), 0: value w (a row of C)
  double w;
};

template <typename T>
__global__ void port_gather_kernel(Geo<T> g, const T *__restrict__ V, int64_t n3, int q,
                                   const PortEdge *__restrict__ pe, int64_t ne, int nports, int transpose,
                                   double *__restrict__ out) {
  extern __shared__ double acc[];
  const int a = blockIdx.x;
  for (int p = threadIdx.x; p < nports; p += blockDim.x) acc[p] = 0;
  __syncthreads();
  const T *v = V + (size_t)a * n3;
  for (int64_t t = threadIdx.x; t < ne; t += blockDim.x) {
    const PortEdge x = pe[t];
    double val = x.w;
    if (x.by_volume) {
      const int c = (int)(x.e / g.nc);
      const int64_t n = x.e - c * g.nc;
      const int idx[3] = {(int)(n % g.nx), (int)((n / g.nx) % g.ny), (int)(n / ((int64_t)g.nx * g.ny))};
      const int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
      const double r = (double)g.rd(c, idx[c]) * (double)g.rdd(a1, idx[a1]) * (double)g.rdd(a2, idx[a2]);
      val = r > 0 ? -x.w / r : 0.0;
    }
    atomicAdd(&acc[x.port], (double)v[x.e] * val);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < nports; p += blockDim.x) {
    if (transpose) out[(size_t)p * q + a] = acc[p];
    else out[(size_t)a * nports + p] = acc[p];
  }
}

template <typename T>
static fdtd_status gram(cudaStream_t s, int64_t nrows, const T *A, int qa, const T *Bm, int qb, const T *w,
                        DevBuf &partial, double *out) {
  if (qa == 0 || qb == 0) return FDTD_OK;
  const int64_t want_slices = std::max<int64_t>(1, (152 * 4) / (((qa + GT - 1) / GT) * ((qb + GT - 1) / GT)));
  int64_t slice = std::max<int64_t>(GK, (nrows + want_slices - 1) / want_slices);
  slice = ((slice + GK - 1) / GK) * GK;
  const int nslice = (int)((nrows + slice - 1) / slice);
  FDTD_CHECK(partial.alloc(sizeof(double) * (size_t)nslice * qa * qb, s));
  dim3 grid((qa + GT - 1) / GT, (qb + GT - 1) / GT, nslice);
  gram_kernel<T><<<grid, 256, 0, s>>>(nrows, A, qa, Bm, qb, w, slice, partial.as<double>());
  FDTD_CHECK(after_launch("gram_kernel"));
  const int n = qa * qb;
  sum_slices_kernel<<<(n + 255) / 256, 256, 0, s>>>(nslice, n, partial.as<double>(), out);
  return after_launch("sum_slices_kernel");
}

fdtd_status gram_native(cudaStream_t s, int64_t n, const float *A, int M, const float *B, int N, double *out) {
  DevBuf partial;
  fdtd_status st = gram<float>(s, n, A, M, B, N, nullptr, partial, out);
  partial.release(s);
  return st;
}

fdtd_status gram_native(cudaStream_t s, int64_t n, const double *A, int M, const double *B, int N, double *out) {
  DevBuf partial;
  fdtd_status st = gram<double>(s, n, A, M, B, N, nullptr, partial, out);
  partial.release(s);
  return st;
}

// G = (G + G^T) / 2 for a q x q row-major matrix: V^T D V is symmetric by
// definition, while the split-precision tensor-core product applies the
// weights to one operand before splitting and so rounds the two triangles
// differently.
__global__ void symmetrize_kernel(int q, double *G) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)q * q) return;
  const int i = (int)(t / q), j = (int)(t % q);
  if (j <= i) return;
  const double a = 0.5 * (G[(int64_t)i * q + j] + G[(int64_t)j * q + i]);
  G[(int64_t)i * q + j] = a;
  G[(int64_t)j * q + i] = a;
}

template <typename T>
static fdtd_status project_t(fdtd_grid *g, const mor_basis *b, cudaStream_t s, mor_model *M) {
  FDTD_CHECK(ensure_edge_props(g, s));
  const int64_t nc = g->nc, n3 = 3 * nc;
  const int q1 = b->q1, q2 = b->q2, m = (int)g->ports.size(), p = (int)g->probes.size();
  M->q1 = q1; M->q2 = q2; M->m = m; M->p = p;
  M->prec = g->prec; M->elem = g->elem; M->stream = s;
  const T *V1 = b->V1.as<T>(), *V2 = b->V2.as<T>();
  DevBuf wts, W, partial;
  FDTD_CHECK(wts.alloc(sizeof(T) * 4 * n3, s));
  const int bl = (int)((nc + 255) / 256);
  diag_weights_kernel<T><<<bl, 256, 0, s>>>(make_geo<T>(g), g->eprops.as<T>(), wts.as<T>());
  FDTD_CHECK(after_launch("diag_weights_kernel"));
  const T *w = wts.as<T>();
  FDTD_CHECK(M->De.alloc(sizeof(double) * std::max(1, q1 * q1), s));
  FDTD_CHECK(M->Dse.alloc(sizeof(double) * std::max(1, q1 * q1), s));
  FDTD_CHECK(M->Dm.alloc(sizeof(double) * std::max(1, q2 * q2), s));
  FDTD_CHECK(M->Dsm.alloc(sizeof(double) * std::max(1, q2 * q2), s));
  FDTD_CHECK(M->K.alloc(sizeof(double) * std::max(1, q1 * q2), s));
  FDTD_CHECK(M->Kp.alloc(sizeof(double) * std::max(1, q1 * q2), s));
  FDTD_CHECK(M->BE.alloc(sizeof(double) * std::max(1, q1 * m), s));
  FDTD_CHECK(M->BH.alloc(sizeof(double) * std::max(1, q2 * m), s));
  FDTD_CHECK(M->CE.alloc(sizeof(double) * std::max(1, p * q1), s));
  FDTD_CHECK(M->sigma.alloc(sizeof(double) * std::max(1, std::min(q1, q2)), s));
  // the five products on the tensor cores when the basis was built with TF32
  // or BF16 Gram-Schmidt products (FP32 grids), else FP32 CUDA cores.  The
  // tensor-core products are split-precision (three passes, gram_tensor_split):
  // one TF32 / BF16 pass would put a 2^-11 / 2^-9 relative error on every
  // entry of the reduced matrices, which the reduced model magnifies to
  // 1e-2 / 7e-2 in its probe waveforms.
  int parith = b->orth;  // FDTDMOR_PROJECT=native / tf32 / bf16 overrides (measurements)
  if (const char *e = getenv("FDTDMOR_PROJECT")) {
    const std::string v(e);
    parith = v == "native" ? MOR_ORTH_NATIVE : v == "tf32" ? MOR_ORTH_TF32 : v == "bf16" ? MOR_ORTH_BF16 : parith;
  }
  const bool tc = sizeof(T) == 4 && parith != MOR_ORTH_NATIVE;
  DevBuf tflag;  // set by a tensor-core pipeline wait that gave up
  if (tc) {
    FDTD_CHECK(tflag.alloc(sizeof(unsigned), s));
    FDTD_CHECK_CUDA(cudaMemsetAsync(tflag.ptr, 0, sizeof(unsigned), s));
  }
  auto G = [&](const T *A, int qa, const T *Bm, int qb, const T *wt, double *out) -> fdtd_status {
    if (tc)
      return gram_tensor_split(s, parith == MOR_ORTH_BF16, n3, reinterpret_cast<const float *>(A), n3, qa,
                               reinterpret_cast<const float *>(Bm), n3, qb, reinterpret_cast<const float *>(wt), out,
                               tflag.as<unsigned>());
    return gram<T>(s, n3, A, qa, Bm, qb, wt, partial, out);
  };
  FDTD_CHECK(G(V1, q1, V1, q1, w + 0 * n3, M->De.as<double>()));
  FDTD_CHECK(G(V1, q1, V1, q1, w + 1 * n3, M->Dse.as<double>()));
  FDTD_CHECK(G(V2, q2, V2, q2, w + 2 * n3, M->Dm.as<double>()));
  FDTD_CHECK(G(V2, q2, V2, q2, w + 3 * n3, M->Dsm.as<double>()));
  if (tc) {
    for (auto pr : {std::make_pair(q1, &M->De), std::make_pair(q1, &M->Dse), std::make_pair(q2, &M->Dm),
                    std::make_pair(q2, &M->Dsm)}) {
      const int64_t nn = (int64_t)pr.first * pr.first;
      if (nn == 0) continue;
      symmetrize_kernel<<<(int)((nn + 255) / 256), 256, 0, s>>>(pr.first, pr.second->as<double>());
      FDTD_CHECK(after_launch("symmetrize_kernel"));
    }
  }
  if (q1 && q2) {
    FDTD_CHECK(W.alloc(sizeof(T) * (size_t)q2 * n3, s));
    dim3 grid(bl, q2);
    kv_kernel<T><<<grid, 256, 0, s>>>(make_geo<T>(g), g->eprops.as<T>(), V2, W.as<T>());
    FDTD_CHECK(after_launch("kv_kernel"));
    FDTD_CHECK(G(V1, q1, W.as<T>(), q2, nullptr, M->K.as<double>()));
  }
  // B~_E (q1 x m) from the source edges, C~_E (p x q1) from the probe edges
  std::vector<PortEdge> src, prb;
  for (int pi = 0; pi < m; ++pi)
    for (size_t e = 0; e < g->ports[pi].cell.size(); ++e)
      src.push_back({g->ports[pi].comp * nc + g->ports[pi].cell[e], pi, 1, g->ports[pi].w[e]});
  for (int pi = 0; pi < p; ++pi)
    for (size_t e = 0; e < g->probes[pi].cell.size(); ++e)
      prb.push_back({g->probes[pi].comp * nc + g->probes[pi].cell[e], pi, 0, g->probes[pi].w[e]});
  DevBuf dsrc, dprb;
  FDTD_CHECK(dsrc.alloc(sizeof(PortEdge) * std::max<size_t>(1, src.size()), s));
  FDTD_CHECK(dprb.alloc(sizeof(PortEdge) * std::max<size_t>(1, prb.size()), s));
  if (!src.empty()) FDTD_CHECK_CUDA(cudaMemcpyAsync(dsrc.ptr, src.data(), sizeof(PortEdge) * src.size(), cudaMemcpyHostToDevice, s));
  if (!prb.empty()) FDTD_CHECK_CUDA(cudaMemcpyAsync(dprb.ptr, prb.data(), sizeof(PortEdge) * prb.size(), cudaMemcpyHostToDevice, s));
  FDTD_CHECK_CUDA(cudaMemsetAsync(M->BH.ptr, 0, sizeof(double) * std::max(1, q2 * m), s));
  if (q1 && m) {
    port_gather_kernel<T><<<q1, 256, sizeof(double) * m, s>>>(make_geo<T>(g), V1, n3, q1, dsrc.as<PortEdge>(), (int64_t)src.size(), m, 0, M->BE.as<double>());
    FDTD_CHECK(after_launch("port_gather_kernel"));
  }
  if (q1 && p) {
    port_gather_kernel<T><<<q1, 256, sizeof(double) * p, s>>>(make_geo<T>(g), V1, n3, q1, dprb.as<PortEdge>(), (int64_t)prb.size(), p, 1, M->CE.as<double>());
    FDTD_CHECK(after_launch("port_gather_kernel"));
  }
  if (tc) {
    unsigned hflag = 0;
    FDTD_CHECK_CUDA(cudaMemcpyAsync(&hflag, tflag.ptr, sizeof(hflag), cudaMemcpyDeviceToHost, s));
    FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
    tflag.release(s);
    FDTD_REQUIRE_STATUS(hflag == 0, FDTD_ETIMEOUT, "mor_project: a bounded tensor-core wait gave up");
  }
  // the unperturbed K~ is also the working K~' until mor_perturb runs
  FDTD_CHECK_CUDA(cudaMemcpyAsync(M->Kp.ptr, M->K.ptr, sizeof(double) * q1 * q2, cudaMemcpyDeviceToDevice, s));
  FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  for (DevBuf *d : {&wts, &W, &partial, &dsrc, &dprb}) d->release(s);
  return FDTD_OK;
}

}  // namespace fdtdmor

using namespace fdtdmor;

extern "C" {

fdtd_status mor_gram(int arith, int64_t n, const float *A, int64_t lda, int M, const float *B, int64_t ldb, int N,
                     const float *w, double *G, fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(A && B && G, "mor_gram: NULL argument");
  FDTD_REQUIRE(n >= 1 && M >= 0 && N >= 0 && lda >= n && ldb >= n, "mor_gram: bad sizes");
  FDTD_REQUIRE(arith >= MOR_ORTH_NATIVE && arith <= MOR_GRAM_BF16X3, "mor_gram: unknown arithmetic %d", arith);
  cudaStream_t s = (cudaStream_t)stream;
  if (arith == MOR_ORTH_NATIVE) {
    FDTD_REQUIRE(lda == n && ldb == n, "mor_gram: the FP32 path needs lda = ldb = n");
    DevBuf partial;
    fdtd_status st = gram<float>(s, n, A, M, B, N, w, partial, G);
    partial.release(s);
    return st;
  }
  DevBuf flag;
  FDTD_CHECK(flag.alloc(sizeof(unsigned), s));
  fdtd_status st = FDTD_OK;
  if (cudaMemsetAsync(flag.ptr, 0, sizeof(unsigned), s) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "memset");
  if (st == FDTD_OK) {
    const bool bf16 = arith == MOR_ORTH_BF16 || arith == MOR_GRAM_BF16X3;
    st = arith >= MOR_GRAM_TF32X3 ? gram_tensor_split(s, bf16, n, A, lda, M, B, ldb, N, w, G, flag.as<unsigned>())
                                  : gram_tensor(s, bf16, n, A, lda, M, B, ldb, N, w, G, flag.as<unsigned>());
  }
  unsigned h = 0;
  if (st == FDTD_OK && cudaMemcpyAsync(&h, flag.ptr, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "flag copy");
  if (st == FDTD_OK && cudaStreamSynchronize(s) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "sync");
  flag.release(s);
  if (st == FDTD_OK && h) {
    set_error("mor_gram: a bounded tensor-core pipeline wait gave up");
    st = FDTD_ETIMEOUT;
  }
  return st;
}

fdtd_status mor_project(fdtd_grid *g, const mor_basis *b, fdtd_stream_t stream, mor_model **out) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(g && b && out, "mor_project: NULL argument");
  FDTD_REQUIRE(b->prec == g->prec && b->n3 == 3 * g->nc, "mor_project: basis does not belong to this grid");
  *out = nullptr;
  mor_model *M = new mor_model();
  fdtd_status st = g->prec == FDTD_F64 ? project_t<double>(g, b, (cudaStream_t)stream, M)
                                       : project_t<float>(g, b, (cudaStream_t)stream, M);
  if (st != FDTD_OK) {
    mor_model_destroy(M);
    return st;
  }
  *out = M;
  return FDTD_OK;
}

}  // extern "C"
