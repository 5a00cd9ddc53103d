// A1: grid and material setup (Sec. II-A, Eq. (matrix)), field access, Eq. (CFL).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "grid_internal.cuh"

namespace fdtdmor {

// Per-axis tables: 1/d, 2/(d[i-1]+d[i]) (0 at i = 0) and the two cell weights
// d[i-1]/(d[i-1]+d[i]), d[i]/(d[i-1]+d[i]) of the edge-average (Sec. II-A reading).
template <typename T>
__global__ void axis_tables_kernel(const double *__restrict__ d, int ntot, T *__restrict__ out,
                                   const int *__restrict__ axis_start) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntot) return;
  int a = (t >= axis_start[1]) + (t >= axis_start[2]);
  int i = t - axis_start[a];
  double di = d[t];
  double dm = (i > 0) ? d[t - 1] : 0.0;
  out[AX_RD * ntot + t] = (T)(1.0 / di);
  out[AX_RDD * ntot + t] = (T)((i > 0) ? 2.0 / (dm + di) : 0.0);
  out[AX_WLO * ntot + t] = (T)((i > 0) ? dm / (dm + di) : 0.0);
  out[AX_WHI * ntot + t] = (T)((i > 0) ? di / (dm + di) : 1.0);
}

// Raw per-material properties in the field type: eps0*eps_r, sig_e, mu0*mu_r, sig_m, pec.
template <typename T>
__global__ void material_table_kernel(const double *__restrict__ raw, int nmat, T *__restrict__ out) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nmat) return;
  out[0 * nmat + m] = (T)(kEps0 * raw[0 * nmat + m]);
  out[1 * nmat + m] = (T)(raw[1 * nmat + m]);
  out[2 * nmat + m] = (T)(kMu0 * raw[2 * nmat + m]);
  out[3 * nmat + m] = (T)(raw[3 * nmat + m]);
  out[4 * nmat + m] = (T)(raw[4 * nmat + m]);
}

// Update coefficients of Eq. (matrix) for one dt, per homogeneous material:
// Ca = (eps/dt - sig/2)/(eps/dt + sig/2), Cb = 1/(eps/dt + sig/2) (zero for PEC),
// Da, Db likewise with mu and sig_m.
template <typename T>
__global__ void coef_table_kernel(const double *__restrict__ raw, int nmat, double dt,
                                  T *__restrict__ out) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nmat) return;
  double eps = kEps0 * raw[0 * nmat + m], sig = raw[1 * nmat + m];
  double mu = kMu0 * raw[2 * nmat + m], sgm = raw[3 * nmat + m];
  bool pec = raw[4 * nmat + m] != 0.0;
  double ae = eps / dt, am = mu / dt;
  double cb = 1.0 / (ae + 0.5 * sig), db = 1.0 / (am + 0.5 * sgm);
  out[0 * nmat + m] = pec ? (T)0 : (T)((ae - 0.5 * sig) * cb);
  out[1 * nmat + m] = pec ? (T)0 : (T)cb;
  out[2 * nmat + m] = (T)((am - 0.5 * sgm) * db);
  out[3 * nmat + m] = (T)db;
}

fdtd_status ensure_coef_table(fdtd_grid *g, double dt, cudaStream_t s) {
  if (g->ctab_dt == dt) return FDTD_OK;
  FDTD_CHECK(g->ctab.alloc((size_t)4 * g->nmat * g->elem, s));
  int th = 128, bl = (g->nmat + th - 1) / th;
  if (g->prec == FDTD_F64)
    coef_table_kernel<double><<<bl, th, 0, s>>>(g->mraw.as<double>(), g->nmat, dt,
                                                g->ctab.as<double>());
  else
    coef_table_kernel<float><<<bl, th, 0, s>>>(g->mraw.as<double>(), g->nmat, dt,
                                               g->ctab.as<float>());
  FDTD_CHECK(after_launch("coef_table_kernel"));
  g->ctab_dt = dt;
  ++g->ctab_version;
  return FDTD_OK;
}

fdtd_status build_tile_lists(fdtd_grid *g, int tx, int ty, cudaStream_t s) {
  TileLists &L = g->lists;
  if (L.tx == tx && L.ty == ty && L.src_ptr.ptr) return FDTD_OK;
  L.tx = tx;
  L.ty = ty;
  L.ntx = (g->nx + tx - 1) / tx;
  L.nty = (g->ny + ty - 1) / ty;
  int ntiles = L.ntx * L.nty;
  auto build = [&](const std::vector<HostPort> &ports, bool halo, DevBuf &ptr, DevBuf &ent,
                   int64_t &count) -> fdtd_status {
    std::vector<std::vector<PortEntry>> per(ntiles);
    for (size_t p = 0; p < ports.size(); ++p) {
      const HostPort &hp = ports[p];
      for (size_t e = 0; e < hp.cell.size(); ++e) {
        int64_t c = hp.cell[e];
        int i = (int)(c % g->nx), j = (int)((c / g->nx) % g->ny), k = (int)(c / ((int64_t)g->nx * g->ny));
        int bx = i / tx, by = j / ty;
        PortEntry pe{};
        pe.k = k;
        pe.comp = (int16_t)hp.comp;
        pe.port = (int32_t)p;
        pe.w = hp.w[e];
        pe.lx = (int16_t)(i - bx * tx);
        pe.ly = (int16_t)(j - by * ty);
        per[by * L.ntx + bx].push_back(pe);
        if (halo && pe.lx == 0 && bx > 0) {  // x-halo column of the left tile
          PortEntry h = pe;
          h.lx = (int16_t)tx;
          per[by * L.ntx + bx - 1].push_back(h);
        }
        if (halo && pe.ly == 0 && by > 0) {  // y-halo row of the tile below
          PortEntry h = pe;
          h.ly = (int16_t)ty;
          per[(by - 1) * L.ntx + bx].push_back(h);
        }
      }
    }
    std::vector<int32_t> hptr(ntiles + 1, 0);
    std::vector<PortEntry> all;
    for (int t = 0; t < ntiles; ++t) {
      std::stable_sort(per[t].begin(), per[t].end(),
                       [](const PortEntry &a, const PortEntry &b) { return a.k < b.k; });
      hptr[t] = (int32_t)all.size();
      all.insert(all.end(), per[t].begin(), per[t].end());
    }
    hptr[ntiles] = (int32_t)all.size();
    count = (int64_t)all.size();
    FDTD_CHECK(ptr.alloc(sizeof(int32_t) * (ntiles + 1), s));
    FDTD_CHECK(ent.alloc(sizeof(PortEntry) * std::max<size_t>(1, all.size()), s));
    FDTD_CHECK_CUDA(cudaMemcpyAsync(ptr.ptr, hptr.data(), sizeof(int32_t) * (ntiles + 1),
                                    cudaMemcpyHostToDevice, s));
    if (!all.empty())
      FDTD_CHECK_CUDA(cudaMemcpyAsync(ent.ptr, all.data(), sizeof(PortEntry) * all.size(),
                                      cudaMemcpyHostToDevice, s));
    // the host vectors die here: make the pageable copies complete first
    FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
    return FDTD_OK;
  };
  FDTD_CHECK(build(g->ports, true, L.src_ptr, L.src, L.nsrc));
  FDTD_CHECK(build(g->probes, false, L.prb_ptr, L.prb, L.nprb));
  return FDTD_OK;
}

static fdtd_status copy_ports(const fdtd_port *in, int n, const fdtd_grid *g,
                              std::vector<HostPort> &out) {
  out.clear();
  for (int p = 0; p < n; ++p) {
    FDTD_REQUIRE(in[p].comp >= 0 && in[p].comp <= 2, "port %d: comp must be 0..2", p);
    FDTD_REQUIRE(in[p].n >= 0 && (in[p].n == 0 || (in[p].cell && in[p].w)),
                 "port %d: missing cell/weight arrays", p);
    HostPort hp;
    hp.comp = in[p].comp;
    for (int64_t e = 0; e < in[p].n; ++e) {
      FDTD_REQUIRE(in[p].cell[e] >= 0 && in[p].cell[e] < g->nc, "port %d: cell index out of range", p);
      hp.cell.push_back(in[p].cell[e]);
      hp.w.push_back(in[p].w[e]);
    }
    out.push_back(std::move(hp));
  }
  return FDTD_OK;
}

// homog_h (one mu_r, sig_m over the materials in use) and the CFL limit of
// Eq. (CFL) from the host material table and spacings.
static void derive_material_props(fdtd_grid *g) {
  double mu0 = -1, sm0 = -1, emin = 1e300;
  g->homog_h = true;
  for (uint16_t i : g->used_mats) {
    if (mu0 < 0) { mu0 = g->mu_r[i]; sm0 = g->sig_m[i]; }
    if (g->mu_r[i] != mu0 || g->sig_m[i] != sm0) g->homog_h = false;
    if (!g->pec[i]) emin = std::min(emin, g->eps_r[i] * g->mu_r[i]);
  }
  if (emin > 1e299) emin = 1.0;
  double dxm = *std::min_element(g->dx.begin(), g->dx.end());
  double dym = *std::min_element(g->dy.begin(), g->dy.end());
  double dzm = *std::min_element(g->dz.begin(), g->dz.end());
  // a single layer between the z plates (nz = 1) is the 2-D TM problem: no
  // update differences along z, so Eq. (CFL) keeps only the x and y terms
  const double zterm = g->nz == 1 ? 0.0 : 1 / (dzm * dzm);
  g->cfl = 1.0 / ((kC0 / std::sqrt(emin)) * std::sqrt(1 / (dxm * dxm) + 1 / (dym * dym) + zterm));
}

// Raw table (eps_r, sig_e, mu_r, sig_m, pec; 5 x nmat doubles) on the device
// into mraw and the field-type table mtab.
static fdtd_status upload_materials(fdtd_grid *g, const double *raw_dev, cudaStream_t s) {
  const int th = 128;
  if (g->prec == FDTD_F64)
    material_table_kernel<double><<<(g->nmat + th - 1) / th, th, 0, s>>>(raw_dev, g->nmat, g->mtab.as<double>());
  else
    material_table_kernel<float><<<(g->nmat + th - 1) / th, th, 0, s>>>(raw_dev, g->nmat, g->mtab.as<float>());
  FDTD_CHECK(after_launch("material_table_kernel"));
  FDTD_CHECK_CUDA(cudaMemcpyAsync(g->mraw.ptr, raw_dev, (size_t)5 * g->nmat * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return FDTD_OK;
}

}  // namespace fdtdmor

using namespace fdtdmor;

extern "C" {

fdtd_status fdtd_grid_set_materials(fdtd_grid *g, int nmat, const double *eps_r, const double *mu_r,
                                    const double *sig_e, const double *sig_m, const uint8_t *pec,
                                    fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(g, "fdtd_grid_set_materials: NULL grid");
  FDTD_REQUIRE(nmat == g->nmat, "fdtd_grid_set_materials: nmat %d differs from the grid's %d", nmat, g->nmat);
  FDTD_REQUIRE(eps_r && mu_r && sig_e && sig_m && pec, "fdtd_grid_set_materials: missing material table");
  for (int i = 0; i < nmat; ++i)
    FDTD_REQUIRE(eps_r[i] > 0 && mu_r[i] > 0 && sig_e[i] >= 0 && sig_m[i] >= 0,
                 "material %d: need eps_r > 0, mu_r > 0, sigma >= 0", i);
  cudaStream_t s = (cudaStream_t)stream;
  g->eps_r.assign(eps_r, eps_r + nmat);
  g->mu_r.assign(mu_r, mu_r + nmat);
  g->sig_e.assign(sig_e, sig_e + nmat);
  g->sig_m.assign(sig_m, sig_m + nmat);
  g->pec.assign(pec, pec + nmat);
  derive_material_props(g);
  std::vector<double> raw;
  raw.insert(raw.end(), g->eps_r.begin(), g->eps_r.end());
  raw.insert(raw.end(), g->sig_e.begin(), g->sig_e.end());
  raw.insert(raw.end(), g->mu_r.begin(), g->mu_r.end());
  raw.insert(raw.end(), g->sig_m.begin(), g->sig_m.end());
  for (int i = 0; i < nmat; ++i) raw.push_back(g->pec[i] ? 1.0 : 0.0);
  DevBuf stage;
  FDTD_CHECK(stage.alloc(raw.size() * sizeof(double), s));
  fdtd_status st = FDTD_OK;
  if (cudaMemcpyAsync(stage.ptr, raw.data(), raw.size() * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "upload materials");
  if (st == FDTD_OK) st = upload_materials(g, stage.as<double>(), s);
  if (st == FDTD_OK && cudaStreamSynchronize(s) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "sync");
  stage.release(s);
  g->ctab_dt = -1;          // coefficient table and edge properties follow the new table
  g->eprops_ready = false;
  return st;
}

fdtd_status fdtd_grid_create(const fdtd_grid_desc *d, int m, const fdtd_port *ports, int p,
                             const fdtd_port *probes, fdtd_stream_t stream, fdtd_grid **out) {
  FDTD_API_RANGE(__func__);
  cudaStream_t s = (cudaStream_t)stream;
  FDTD_REQUIRE(d && out, "fdtd_grid_create: NULL descriptor or output");
  *out = nullptr;
  FDTD_REQUIRE(d->nx >= 1 && d->ny >= 1 && d->nz >= 1, "grid dimensions must be >= 1");
  FDTD_REQUIRE((int64_t)d->nx * d->ny * d->nz < ((int64_t)1 << 40), "grid too large");
  FDTD_REQUIRE(d->dx && d->dy && d->dz && d->mat_id, "missing spacing or material-id array");
  FDTD_REQUIRE(d->nmat >= 1 && d->nmat <= 65535, "nmat must be 1..65535");
  FDTD_REQUIRE(d->eps_r && d->mu_r && d->sig_e && d->sig_m && d->pec, "missing material table");
  FDTD_REQUIRE(d->prec == FDTD_F32 || d->prec == FDTD_F64, "prec must be FDTD_F32 or FDTD_F64");
  FDTD_REQUIRE(m >= 0 && p >= 0 && (m == 0 || ports) && (p == 0 || probes), "bad port lists");
  fdtd_grid *g = new fdtd_grid();
  g->nx = d->nx; g->ny = d->ny; g->nz = d->nz;
  g->nc = (int64_t)d->nx * d->ny * d->nz;
  g->prec = d->prec;
  g->elem = d->prec == FDTD_F64 ? 8 : 4;
  g->nmat = d->nmat;
  g->id_bytes = d->nmat <= 255 ? 1 : 2;   // the largest id value is kept free as a sentinel
  g->create_stream = s;
  auto fail = [&](fdtd_status st) { fdtd_grid_destroy(g); return st; };
  g->dx.assign(d->dx, d->dx + d->nx);
  g->dy.assign(d->dy, d->dy + d->ny);
  g->dz.assign(d->dz, d->dz + d->nz);
  for (double v : g->dx) if (!(v > 0)) { set_error("dx must be > 0"); return fail(FDTD_EINVAL); }
  for (double v : g->dy) if (!(v > 0)) { set_error("dy must be > 0"); return fail(FDTD_EINVAL); }
  for (double v : g->dz) if (!(v > 0)) { set_error("dz must be > 0"); return fail(FDTD_EINVAL); }
  g->eps_r.assign(d->eps_r, d->eps_r + d->nmat);
  g->mu_r.assign(d->mu_r, d->mu_r + d->nmat);
  g->sig_e.assign(d->sig_e, d->sig_e + d->nmat);
  g->sig_m.assign(d->sig_m, d->sig_m + d->nmat);
  g->pec.assign(d->pec, d->pec + d->nmat);
  for (int i = 0; i < d->nmat; ++i) {
    if (!(g->eps_r[i] > 0 && g->mu_r[i] > 0 && g->sig_e[i] >= 0 && g->sig_m[i] >= 0)) {
      set_error("material %d: need eps_r > 0, mu_r > 0, sigma >= 0", i);
      return fail(FDTD_EINVAL);
    }
  }
  std::vector<uint8_t> seen(d->nmat, 0);
  for (int64_t c = 0; c < g->nc; ++c) {
    if (d->mat_id[c] >= d->nmat) {
      set_error("mat_id[%lld] = %d >= nmat", (long long)c, (int)d->mat_id[c]);
      return fail(FDTD_EINVAL);
    }
    seen[d->mat_id[c]] = 1;
  }
  for (int i = 0; i < d->nmat; ++i)
    if (seen[i]) g->used_mats.push_back((uint16_t)i);
  derive_material_props(g);
  fdtd_status st;
  if ((st = copy_ports(ports, m, g, g->ports)) != FDTD_OK) return fail(st);
  if ((st = copy_ports(probes, p, g, g->probes)) != FDTD_OK) return fail(st);

  // device state
  size_t fbytes = (size_t)6 * g->nc * g->elem;
  for (int b = 0; b < 2; ++b) {
    if ((st = g->fields[b].alloc(fbytes, s)) != FDTD_OK) return fail(st);
  }
  if (cudaMemsetAsync(g->fields[0].ptr, 0, fbytes, s) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "memset"));
  if ((st = g->mat.alloc((size_t)g->nc * g->id_bytes, s)) != FDTD_OK) return fail(st);
  if ((st = g->errflag.alloc(sizeof(unsigned), s)) != FDTD_OK) return fail(st);
  if (cudaMemsetAsync(g->errflag.ptr, 0, sizeof(unsigned), s) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "memset"));
  if (g->id_bytes == 2) {
    if (cudaMemcpyAsync(g->mat.ptr, d->mat_id, g->nc * 2, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return fail(cuda_fail(cudaGetLastError(), "upload mat_id"));
  } else {
    std::vector<uint8_t> m8(g->nc);
    for (int64_t c = 0; c < g->nc; ++c) m8[c] = (uint8_t)d->mat_id[c];
    if (cudaMemcpyAsync(g->mat.ptr, m8.data(), g->nc, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return fail(cuda_fail(cudaGetLastError(), "upload mat_id"));
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "sync"));
  }
  // spacings and material raw table go through one staging upload
  int ntot = g->nx + g->ny + g->nz;
  std::vector<double> stage;
  stage.insert(stage.end(), g->dx.begin(), g->dx.end());
  stage.insert(stage.end(), g->dy.begin(), g->dy.end());
  stage.insert(stage.end(), g->dz.begin(), g->dz.end());
  size_t raw_off = stage.size();
  stage.insert(stage.end(), g->eps_r.begin(), g->eps_r.end());
  stage.insert(stage.end(), g->sig_e.begin(), g->sig_e.end());
  stage.insert(stage.end(), g->mu_r.begin(), g->mu_r.end());
  stage.insert(stage.end(), g->sig_m.begin(), g->sig_m.end());
  for (int i = 0; i < d->nmat; ++i) stage.push_back(g->pec[i] ? 1.0 : 0.0);
  int starts[3] = {0, g->nx, g->nx + g->ny};
  DevBuf dstage, dstarts;
  if ((st = dstage.alloc(stage.size() * sizeof(double), s)) != FDTD_OK) return fail(st);
  if ((st = dstarts.alloc(sizeof(starts), s)) != FDTD_OK) return fail(st);
  cudaMemcpyAsync(dstage.ptr, stage.data(), stage.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dstarts.ptr, starts, sizeof(starts), cudaMemcpyHostToDevice, s);
  if ((st = g->axis.alloc((size_t)AX_COUNT * ntot * g->elem, s)) != FDTD_OK) return fail(st);
  if ((st = g->mtab.alloc((size_t)5 * g->nmat * g->elem, s)) != FDTD_OK) return fail(st);
  if ((st = g->mraw.alloc((size_t)5 * g->nmat * sizeof(double), s)) != FDTD_OK) return fail(st);
  int th = 128;
  double *raw = dstage.as<double>() + raw_off;
  if (g->prec == FDTD_F64)
    axis_tables_kernel<double><<<(ntot + th - 1) / th, th, 0, s>>>(dstage.as<double>(), ntot, g->axis.as<double>(), dstarts.as<int>());
  else
    axis_tables_kernel<float><<<(ntot + th - 1) / th, th, 0, s>>>(dstage.as<double>(), ntot, g->axis.as<float>(), dstarts.as<int>());
  if ((st = after_launch("axis_tables_kernel")) != FDTD_OK) return fail(st);
  if ((st = upload_materials(g, raw, s)) != FDTD_OK) return fail(st);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "grid setup"));
  dstage.release(s);
  dstarts.release(s);
  *out = g;
  return FDTD_OK;
}

fdtd_status fdtd_grid_destroy(fdtd_grid *g) {
  if (!g) return FDTD_OK;
  cudaStream_t s = g->create_stream;
  cudaStreamSynchronize(s);
  for (auto &b : g->fields) b.release(s);
  g->mat.release(s);
  g->axis.release(s);
  g->mtab.release(s);
  g->mraw.release(s);
  g->ctab.release(s);
  g->lists.src_ptr.release(s);
  g->lists.src.release(s);
  g->lists.prb_ptr.release(s);
  g->lists.prb.release(s);
  g->u_stage.release(s);
  g->y_stage.release(s);
  g->eprops.release(s);
  g->errflag.release(s);
  g->uflag.release(s);
  g->emat.release(s);
  g->ecoef.release(s);
  g->gsync.release(s);
  g->u_graph.release(s);
  g->flat_src.release(s);
  g->flat_prb.release(s);
  g->fix_off.release(s);
  g->fix_fac.release(s);
  g->fix_port.release(s);
  g->y_graph.release(s);
  for (auto &x : g->ygraph)
    if (x) cudaGraphExecDestroy(x);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  cudaStreamSynchronize(s);
  delete g;
  return FDTD_OK;
}

double fdtd_cfl_dt(const fdtd_grid *g) { return g ? g->cfl : -1.0; }

fdtd_status fdtd_check(fdtd_grid *g, fdtd_stream_t stream) {
  FDTD_REQUIRE(g, "fdtd_check: NULL grid");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned h = 0;
  FDTD_CHECK_CUDA(cudaMemcpyAsync(&h, g->errflag.ptr, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  if (h) {
    FDTD_CHECK_CUDA(cudaMemsetAsync(g->errflag.ptr, 0, sizeof(unsigned), s));
    if (h & 3u) {
      set_error("a bounded device-side wait of the stepping kernel gave up; the fields are not valid");
      return FDTD_ETIMEOUT;
    }
    if (h & 16u) {
      set_error("an index check of the checked build failed (a port-list entry outside the grid); the fields are not valid");
      return FDTD_ECUDA;
    }
    set_error("the field watchdog fired: %s", (h & 4u) ? "NaN or Inf in the fields" : "field energy grew beyond the limit");
    return FDTD_EUNSTABLE;
  }
  return FDTD_OK;
}

fdtd_status fdtd_fields_get(const fdtd_grid *g, void *fields6, fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(g && fields6, "fdtd_fields_get: NULL argument");
  FDTD_CHECK_CUDA(cudaMemcpyAsync(fields6, g->fields[g->cur].ptr, (size_t)6 * g->nc * g->elem,
                                  cudaMemcpyDefault, (cudaStream_t)stream));
  return FDTD_OK;
}

fdtd_status fdtd_planes_get(const fdtd_grid *g, int k0, int nk, void *dst, fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(g && dst, "fdtd_planes_get: NULL argument");
  FDTD_REQUIRE(k0 >= 0 && nk >= 0 && k0 + nk <= g->nz, "fdtd_planes_get: planes [%d, %d) outside 0..%d", k0, k0 + nk,
               g->nz);
  const size_t plane = (size_t)g->nx * g->ny * g->elem, chunk = plane * nk;
  const char *src = static_cast<const char *>(g->fields[g->cur].ptr);
  for (int c = 0; c < 6; ++c)
    FDTD_CHECK_CUDA(cudaMemcpyAsync(static_cast<char *>(dst) + c * chunk, src + (size_t)c * g->nc * g->elem + k0 * plane,
                                    chunk, cudaMemcpyDefault, (cudaStream_t)stream));
  return FDTD_OK;
}

fdtd_status fdtd_planes_set(fdtd_grid *g, int k0, int nk, const void *src, fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(g && src, "fdtd_planes_set: NULL argument");
  FDTD_REQUIRE(k0 >= 0 && nk >= 0 && k0 + nk <= g->nz, "fdtd_planes_set: planes [%d, %d) outside 0..%d", k0, k0 + nk,
               g->nz);
  const size_t plane = (size_t)g->nx * g->ny * g->elem, chunk = plane * nk;
  char *dst = static_cast<char *>(g->fields[g->cur].ptr);
  for (int c = 0; c < 6; ++c)
    FDTD_CHECK_CUDA(cudaMemcpyAsync(dst + (size_t)c * g->nc * g->elem + k0 * plane,
                                    static_cast<const char *>(src) + c * chunk, chunk, cudaMemcpyDefault,
                                    (cudaStream_t)stream));
  return FDTD_OK;
}

fdtd_status fdtd_fields_set(fdtd_grid *g, const void *fields6, fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(g && fields6, "fdtd_fields_set: NULL argument");
  FDTD_CHECK_CUDA(cudaMemcpyAsync(g->fields[g->cur].ptr, fields6, (size_t)6 * g->nc * g->elem,
                                  cudaMemcpyDefault, (cudaStream_t)stream));
  return FDTD_OK;
}

}  // extern "C"
