// A12: gradient of a probe loss with respect to the per-cell relative
// permittivity, by the discrete adjoint of the leap-frog (not in the paper;
// the method's full-order recursion of Eq. (matrix) differentiated exactly).
//
// Forward step n (per-volume form, all operators diagonal except the curls):
//   E^{n+1} = Ca E^n + Cb (curlH H^{n+1/2} - w u^{n+1}),
//   H^{n+3/2} = Da H^{n+1/2} - Db curlE E^{n+1},      y^n = P E^{n+1}.
// With curlH = V_e^-1 K and curlE = V_h^-1 K^T (K the integer-length curl
// incidence), the adjoint variables scaled as e^ = Cb ebar / V_e and
// h^ = -Db hbar / V_h obey, backwards in n,
//   e^_{n+1} = Ca e^_{n+2} + Cb (curlH h^_{n+3/2} + P^T ybar^n / V_e),
//   h^_{n+1/2} = Da h^_{n+3/2} - Db curlE e^_{n+1},
// which is the forward step itself with the probes as sources of weight
// -w / V_e driven by ybar^n = dL/dy^n: the adjoint run reuses the leap-frog
// kernels.  Since Ca + sigma Cb = 1, d E^{n+1} / d eps_e = -(Cb/dt)(E^{n+1} - E^n),
// so dL/d eps_e = -sum_n (V_e/dt) e^_{n+1} (E^{n+1} - E^n), and the edge
// permittivity is the area-weighted mean of its four cells (eps0 eps_r).
//
// Memory: the forward states are recomputed from K checkpoints of the full
// state (K = ceil(sqrt(nsteps)) by default); each segment of c steps stores its
// c + 1 E fields, then the adjoint runs back through it.  The per-edge products
// are summed in the field type within a segment and added into an FP64
// per-edge gradient at the end of each segment.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "grid_internal.cuh"
#include "mor_internal.cuh"

namespace fdtdmor {

fdtd_status yee_run(fdtd_grid *g, double dt, int64_t nsteps, const void *u, void *y, int reset_fields,
                    cudaStream_t s);

// gseg[e] += -(V_e/dt) e^[e] (E1[e] - E0[e]) over the 3 nc E edges.
template <typename T>
__global__ void adj_grad_step_kernel(const T *__restrict__ ax, int nx, int ny, int nz, int64_t nc,
                                     const T *__restrict__ eadj, const T *__restrict__ e1,
                                     const T *__restrict__ e0, double inv_dt, T *__restrict__ gseg) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= nc) return;
  const unsigned u = (unsigned)(n % nx);
  const int64_t q = n / nx;
  const int i = (int)u, j = (int)(q % ny), k = (int)(q / ny);
  // V_e = 1 / (rd_c rdd_a rdd_b) in the field type: FP64 divisions per edge
  // made this pass FP64-throughput-bound (1.1 ms per step on 384x384x64)
  const int ntot = nx + ny + nz;
  const int idx[3] = {i, nx + j, nx + ny + k};
  T rd[3], rdd[3];
  for (int a = 0; a < 3; ++a) {
    rd[a] = __ldg(ax + AX_RD * ntot + idx[a]);
    rdd[a] = __ldg(ax + AX_RDD * ntot + idx[a]);
  }
  const T idt = (T)inv_dt;
  for (int c = 0; c < 3; ++c) {
    const int64_t e = c * nc + n;
    const T d = e1[e] - e0[e];
    if (d == T(0)) continue;
    const T den = rd[c] * rdd[(c + 1) % 3] * rdd[(c + 2) % 3];
    if (den == T(0)) continue;  // wall edge: no volume
    gseg[e] += -(idt / den) * eadj[e] * d;
  }
}

// gedge[e] += gseg[e] (FP64), gseg[e] = 0.
template <typename T>
__global__ void adj_flush_kernel(int64_t n3, T *__restrict__ gseg, double *__restrict__ gedge) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n3) return;
  gedge[e] += (double)gseg[e];
  gseg[e] = T(0);
}

// Per cell: dL/d eps_r = eps0 sum over the 12 E edges around the cell of the
// edge gradient times the cell's area weight in that edge's average; per
// material: the sum over its cells (lanes of a warp holding the same id add
// their values first, then one atomic per id).
template <typename T, typename ID>
__global__ void adj_cell_kernel(const T *__restrict__ ax, int nx, int ny, int nz, int64_t nc,
                                const double *__restrict__ gedge, const ID *__restrict__ mat,
                                double *__restrict__ gcell, double *__restrict__ gmat) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double val = 0.0;
  unsigned id = 0xffffffffu;
  if (n < nc) {
    const int64_t q = n / nx;
    const int i = (int)(n % nx), j = (int)(q % ny), k = (int)(q / ny);
    const int ntot = nx + ny + nz;
    auto wlo = [&](int t) { return (double)__ldg(ax + AX_WLO * ntot + t); };
    auto whi = [&](int t) { return (double)__ldg(ax + AX_WHI * ntot + t); };
    auto at = [&](int c, int ii, int jj, int kk) { return gedge[c * nc + ((int64_t)kk * ny + jj) * nx + ii]; };
    double s = 0.0;
    // the cell is the upper neighbour of the edge at its own index and the
    // lower neighbour of the edge one index up
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        {  // Ex edges at (i, j + a, k + b): transverse axes y, z
          const int jj = j + a, kk = k + b;
          if (jj < ny && kk < nz)
            s += (a ? wlo(nx + jj) : whi(nx + jj)) * (b ? wlo(nx + ny + kk) : whi(nx + ny + kk)) * at(0, i, jj, kk);
        }
        {  // Ey edges at (i + a, j, k + b): transverse axes x, z
          const int ii = i + a, kk = k + b;
          if (ii < nx && kk < nz)
            s += (a ? wlo(ii) : whi(ii)) * (b ? wlo(nx + ny + kk) : whi(nx + ny + kk)) * at(1, ii, j, kk);
        }
        {  // Ez edges at (i + a, j + b, k): transverse axes x, y
          const int ii = i + a, jj = j + b;
          if (ii < nx && jj < ny)
            s += (a ? wlo(ii) : whi(ii)) * (b ? wlo(nx + jj) : whi(nx + jj)) * at(2, ii, jj, k);
        }
      }
    val = kEps0 * s;
    if (gcell) gcell[n] = val;
    id = (unsigned)mat[n];
  }
  if (!gmat) return;
  const unsigned grp = __match_any_sync(0xffffffffu, id);
  const int lane = threadIdx.x & 31, leader = __ffs(grp) - 1;
  double sum = 0.0;
  for (unsigned m = grp; m; m &= m - 1) sum += __shfl_sync(grp, val, __ffs(m) - 1);
  if (lane == leader && id != 0xffffffffu) atomicAdd(gmat + id, sum);
}

// Swaps the grid's state, port lists and tile lists with the adjoint run's
// for the lifetime of the object.
struct AdjointView {
  fdtd_grid *g;
  DevBuf *fields;
  int *cur;
  TileLists *lists;
  std::vector<HostPort> *ports, *probes;
  DevBuf fsrc, fprb;             // the adjoint run's flat port lists (fused z-march form)
  int nfsrc = 0, nfprb = 0;
  bool fready = false;
  DevBuf xoff, xfac, xport;      // and its gathered source terms
  int nx_ = 0;
  int64_t xver = -1;
  bool xone = false;
  AdjointView(fdtd_grid *g_, DevBuf *f, int *c, TileLists *l, std::vector<HostPort> *pt, std::vector<HostPort> *pb)
      : g(g_), fields(f), cur(c), lists(l), ports(pt), probes(pb) {
    swap_all();
  }
  ~AdjointView() {
    swap_all();
    fsrc.release(g->create_stream);
    fprb.release(g->create_stream);
    xoff.release(g->create_stream);
    xfac.release(g->create_stream);
    xport.release(g->create_stream);
  }
  void swap_all() {
    std::swap(g->flat_src, fsrc);
    std::swap(g->flat_prb, fprb);
    std::swap(g->nflat_src, nfsrc);
    std::swap(g->nflat_prb, nfprb);
    std::swap(g->flat_ready, fready);
    std::swap(g->fix_off, xoff);
    std::swap(g->fix_fac, xfac);
    std::swap(g->fix_port, xport);
    std::swap(g->nfix, nx_);
    std::swap(g->fix_version, xver);
    std::swap(g->fix_one, xone);
    std::swap(g->fields[0], fields[0]);
    std::swap(g->fields[1], fields[1]);
    std::swap(g->cur, *cur);
    std::swap(g->lists, *lists);
    std::swap(g->ports, *ports);
    std::swap(g->probes, *probes);
  }
};

template <typename T>
static fdtd_status edges_to_cells_t(fdtd_grid *g, const double *gedge, double *gcell, double *gmat, cudaStream_t s) {
  if (gmat) FDTD_CHECK_CUDA(cudaMemsetAsync(gmat, 0, (size_t)g->nmat * sizeof(double), s));
  const int nb1 = (int)((g->nc + 255) / 256);
  const T *ax = g->axis.as<T>();
  if (g->id_bytes == 1)
    adj_cell_kernel<T, uint8_t><<<nb1, 256, 0, s>>>(ax, g->nx, g->ny, g->nz, g->nc, gedge, g->mat.as<uint8_t>(), gcell,
                                                    gmat);
  else
    adj_cell_kernel<T, uint16_t><<<nb1, 256, 0, s>>>(ax, g->nx, g->ny, g->nz, g->nc, gedge, g->mat.as<uint16_t>(),
                                                     gcell, gmat);
  return after_launch("adj_cell_kernel");
}

fdtd_status edges_to_cells(fdtd_grid *g, const double *gedge, double *gcell, double *gmat, cudaStream_t s) {
  return g->prec == FDTD_F64 ? edges_to_cells_t<double>(g, gedge, gcell, gmat, s)
                             : edges_to_cells_t<float>(g, gedge, gcell, gmat, s);
}

template <typename T>
static fdtd_status adjoint_t(fdtd_grid *g, double dt, int64_t T_, const void *u, const void *dldy, int ncheck,
                             double *gcell, double *gmat, cudaStream_t s) {
  const int m = (int)g->ports.size(), p = (int)g->probes.size();
  const int64_t nc = g->nc, n3 = 3 * nc, n6 = 6 * nc;
  const size_t es = sizeof(T);
  int64_t K = ncheck > 0 ? ncheck : (int64_t)std::ceil(std::sqrt((double)T_));
  K = std::max<int64_t>(1, std::min(K, T_));
  const int64_t c = (T_ + K - 1) / K;
  K = (T_ + c - 1) / c;

  DevBuf ckpt, seg, gseg, gedge, yscr;
  struct Release {
    std::vector<DevBuf *> b;
    cudaStream_t s;
    ~Release() { for (auto *x : b) x->release(s); }
  } rel{{&ckpt, &seg, &gseg, &gedge, &yscr}, s};
  FDTD_CHECK(ckpt.alloc((size_t)K * n6 * es, s));
  FDTD_CHECK(seg.alloc((size_t)(c + 1) * n3 * es, s));
  FDTD_CHECK(gseg.alloc((size_t)n3 * es, s));
  FDTD_CHECK(gedge.alloc((size_t)n3 * sizeof(double), s));
  if (p) FDTD_CHECK(yscr.alloc((size_t)c * p * es, s));
  FDTD_CHECK_CUDA(cudaMemsetAsync(gseg.ptr, 0, (size_t)n3 * es, s));
  FDTD_CHECK_CUDA(cudaMemsetAsync(gedge.ptr, 0, (size_t)n3 * sizeof(double), s));

  // adjoint run: its own two state buffers, the probes as sources of weight
  // -w / V_e, no probes
  DevBuf afields[2];
  struct ReleaseF {
    DevBuf *f;
    cudaStream_t s;
    ~ReleaseF() { f[0].release(s); f[1].release(s); }
  } relf{afields, s};
  FDTD_CHECK(afields[0].alloc((size_t)n6 * es, s));
  FDTD_CHECK(afields[1].alloc((size_t)n6 * es, s));
  FDTD_CHECK_CUDA(cudaMemsetAsync(afields[0].ptr, 0, (size_t)n6 * es, s));
  int acur = 0;
  TileLists alists;
  struct ReleaseL {
    TileLists *l;
    cudaStream_t s;
    ~ReleaseL() { l->src_ptr.release(s); l->src.release(s); l->prb_ptr.release(s); l->prb.release(s); }
  } rell{&alists, s};
  std::vector<HostPort> aports, aprobes;
  auto dual = [](const std::vector<double> &d, int t) { return t > 0 ? 0.5 * (d[t - 1] + d[t]) : 0.5 * d[0]; };
  for (const HostPort &hp : g->probes) {
    HostPort a = hp;
    for (size_t q = 0; q < hp.cell.size(); ++q) {
      const int64_t cell = hp.cell[q];
      const int i = (int)(cell % g->nx), j = (int)((cell / g->nx) % g->ny), k = (int)(cell / ((int64_t)g->nx * g->ny));
      double v;
      if (hp.comp == 0) v = g->dx[i] * dual(g->dy, j) * dual(g->dz, k);
      else if (hp.comp == 1) v = dual(g->dx, i) * g->dy[j] * dual(g->dz, k);
      else v = dual(g->dx, i) * dual(g->dy, j) * g->dz[k];
      a.w[q] = -hp.w[q] / v;
    }
    aports.push_back(std::move(a));
  }

  // forward with checkpoints
  FDTD_CHECK_CUDA(cudaMemsetAsync(g->fields[g->cur].ptr, 0, (size_t)n6 * es, s));
  for (int64_t sg = 0; sg < K; ++sg) {
    const int64_t n0 = sg * c, len = std::min(c, T_ - n0);
    FDTD_CHECK_CUDA(cudaMemcpyAsync(ckpt.as<T>() + sg * n6, g->fields[g->cur].ptr, (size_t)n6 * es,
                                    cudaMemcpyDeviceToDevice, s));
    FDTD_CHECK(yee_run(g, dt, len, u ? static_cast<const T *>(u) + n0 * m : nullptr, p ? yscr.ptr : nullptr, 0, s));
  }

  const T *ax = g->axis.as<T>();
  const int th = 256;
  const int nb1 = (int)((nc + th - 1) / th), nb3 = (int)((n3 + th - 1) / th);
  for (int64_t sg = K - 1; sg >= 0; --sg) {
    const int64_t n0 = sg * c, len = std::min(c, T_ - n0);
    // recompute the segment, keeping E^{n0} .. E^{n0+len}
    FDTD_CHECK_CUDA(cudaMemcpyAsync(g->fields[g->cur].ptr, ckpt.as<T>() + sg * n6, (size_t)n6 * es,
                                    cudaMemcpyDeviceToDevice, s));
    FDTD_CHECK_CUDA(cudaMemcpyAsync(seg.ptr, g->fields[g->cur].ptr, (size_t)n3 * es, cudaMemcpyDeviceToDevice, s));
    for (int64_t t = 0; t < len; ++t) {
      FDTD_CHECK(yee_run(g, dt, 1, u ? static_cast<const T *>(u) + (n0 + t) * m : nullptr, p ? yscr.ptr : nullptr,
                         0, s));
      FDTD_CHECK_CUDA(cudaMemcpyAsync(seg.as<T>() + (t + 1) * n3, g->fields[g->cur].ptr, (size_t)n3 * es,
                                      cudaMemcpyDeviceToDevice, s));
    }
    // adjoint steps back through the segment
    {
      AdjointView view(g, afields, &acur, &alists, &aports, &aprobes);
      for (int64_t t = len - 1; t >= 0; --t) {
        const int64_t n = n0 + t;
        FDTD_CHECK(yee_run(g, dt, 1, p ? static_cast<const T *>(dldy) + n * p : nullptr, nullptr, 0, s));
        adj_grad_step_kernel<T><<<nb1, th, 0, s>>>(ax, g->nx, g->ny, g->nz, nc, g->fields[g->cur].as<T>(),
                                                   seg.as<T>() + (t + 1) * n3, seg.as<T>() + t * n3, 1.0 / dt,
                                                   gseg.as<T>());
        FDTD_CHECK(after_launch("adj_grad_step_kernel"));
      }
    }
    adj_flush_kernel<T><<<nb3, th, 0, s>>>(n3, gseg.as<T>(), gedge.as<double>());
    FDTD_CHECK(after_launch("adj_flush_kernel"));
  }
  FDTD_CHECK_CUDA(cudaMemsetAsync(g->fields[g->cur].ptr, 0, (size_t)n6 * es, s));
  FDTD_CHECK(edges_to_cells(g, gedge.as<double>(), gcell, gmat, s));
  // the buffers are released on s after the last kernel that reads them
  return FDTD_OK;
}

}  // namespace fdtdmor

using namespace fdtdmor;

extern "C" {

fdtd_status fdtd_adjoint(fdtd_grid *g, double dt, int64_t nsteps, const void *u, const void *dloss_dy,
                         int ncheckpoints, double *grad_eps_cell, double *grad_eps_mat, fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(g, "fdtd_adjoint: NULL grid");
  FDTD_REQUIRE(dt > 0 && nsteps >= 1, "fdtd_adjoint: need dt > 0 and nsteps >= 1");
  FDTD_REQUIRE(g->ports.empty() || u, "fdtd_adjoint: u is required when the grid has sources");
  FDTD_REQUIRE(g->probes.empty() || dloss_dy, "fdtd_adjoint: dloss_dy is required when the grid has probes");
  FDTD_REQUIRE(grad_eps_cell || grad_eps_mat, "fdtd_adjoint: no output");
  FDTD_REQUIRE(ncheckpoints >= 0, "fdtd_adjoint: ncheckpoints must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  if (g->prec == FDTD_F64) return adjoint_t<double>(g, dt, nsteps, u, dloss_dy, ncheckpoints, grad_eps_cell,
                                                    grad_eps_mat, s);
  return adjoint_t<float>(g, dt, nsteps, u, dloss_dy, ncheckpoints, grad_eps_cell, grad_eps_mat, s);
}

}  // extern "C"
