// A2: full-order Yee leap-frog of Eq. (matrix) / Eq. (MNAform), one fused
// kernel per time step.
//
// Each CTA owns an xy tile of TX x TY cells and marches up a chunk of z planes.
// For plane k it stages H^{n+1/2}[k] (tile plus a one-cell halo) and the cell
// material ids in shared memory, computes E^{n+1}[k] on the tile plus its +x/+y
// halo (the halo values are recomputed redundantly instead of exchanged), adds
// the sources, then computes H^{n+3/2}[k-1] from E^{n+1}[k-1] and E^{n+1}[k].
// Reads E^n, H^{n+1/2} from one buffer and writes E^{n+1}, H^{n+3/2} to the
// other (ping-pong), so every field value is read once and written once per
// step: 48 B (f32) or 96 B (f64) of field traffic per cell-update.
//
// Per edge, (Ca, Cb) come from the per-material table when the cells around
// the edge share a material, else from the area-weighted eps/sigma of those
// cells (the non-uniform, inhomogeneous reading of Sec. II-A).
#include <algorithm>

#include <cstring>
#include <string>

#include "common.cuh"
#include "grid_internal.cuh"
#include "yee_internal.cuh"

namespace fdtdmor {

constexpr int YTX = 32, YTY = 8, YNT = YTX * YTY;
constexpr int YEX = YTX + 1, YEY = YTY + 1;   // E region: tile + high halo
constexpr int YHX = YTX + 2, YHY = YTY + 2;   // H / id region: tile + both halos

template <typename T, typename ID>
struct YeeSmem {
  T H[3][3][YHY][YHX];   // H^{n+1/2}, three plane slots (k % 3)
  T E[2][3][YEY][YEX];   // E^{n+1}, two plane slots (k & 1)
  ID M[4][YHY][YHX];     // material ids, four plane slots (k & 3)
  int rng[2];            // this plane's source range
};

// (Ca, Cb) of E component c at extended-region position (lx, ly) of plane k.
template <typename T, typename ID>
__device__ __forceinline__ void e_coef_at(const YeeArgs<T, ID> &a, const YeeSmem<T, ID> &sm, int c,
                                          int lx, int ly, int i, int j, int k, T &ca, T &cb) {
  const int ntot = a.nx + a.ny + a.nz;
  const int hx = lx + 1, hy = ly + 1;
  const int mk = k & 3, mkm = (k + 3) & 3;  // planes k and k-1
  if (c == 0) {
    if (j == 0 || k == 0) { ca = cb = T(0); return; }
    e_coef(a, sm.M[mkm][hy - 1][hx], sm.M[mkm][hy][hx], sm.M[mk][hy - 1][hx], sm.M[mk][hy][hx],
           axv(a.ax, ntot, AX_WLO, a.nx + j), axv(a.ax, ntot, AX_WHI, a.nx + j),
           axv(a.ax, ntot, AX_WLO, a.nx + a.ny + k), axv(a.ax, ntot, AX_WHI, a.nx + a.ny + k), ca, cb);
  } else if (c == 1) {
    if (i == 0 || k == 0) { ca = cb = T(0); return; }
    e_coef(a, sm.M[mkm][hy][hx - 1], sm.M[mkm][hy][hx], sm.M[mk][hy][hx - 1], sm.M[mk][hy][hx],
           axv(a.ax, ntot, AX_WLO, i), axv(a.ax, ntot, AX_WHI, i),
           axv(a.ax, ntot, AX_WLO, a.nx + a.ny + k), axv(a.ax, ntot, AX_WHI, a.nx + a.ny + k), ca, cb);
  } else {
    if (i == 0 || j == 0) { ca = cb = T(0); return; }
    e_coef(a, sm.M[mk][hy - 1][hx - 1], sm.M[mk][hy - 1][hx], sm.M[mk][hy][hx - 1], sm.M[mk][hy][hx],
           axv(a.ax, ntot, AX_WLO, i), axv(a.ax, ntot, AX_WHI, i),
           axv(a.ax, ntot, AX_WLO, a.nx + j), axv(a.ax, ntot, AX_WHI, a.nx + j), ca, cb);
  }
}

template <typename T, typename ID, bool HOMOG_H>
__global__ void __launch_bounds__(YNT) yee_fused_kernel(YeeArgs<T, ID> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  YeeSmem<T, ID> &sm = *reinterpret_cast<YeeSmem<T, ID> *>(smem_raw);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * YTX + tx;
  const int i0 = blockIdx.x * YTX, j0 = blockIdx.y * YTY;
  const int k0 = blockIdx.z * a.kchunk;
  if (k0 >= a.nz) return;
  const int k1 = min(a.nz, k0 + a.kchunk);
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t nc = a.nc;
  const int ntot = nx + ny + nz;
  const int tile = blockIdx.y * gridDim.x + blockIdx.x;
  const int s_beg = a.src_ptr[tile], s_end = a.src_ptr[tile + 1];
  const int p_beg = a.prb_ptr[tile], p_end = a.prb_ptr[tile + 1];

  auto load_plane = [&](int k) {  // H^{n+1/2}[k] and ids of plane k into their slots
    const int hs = ((k % 3) + 3) % 3, ms = k & 3;
    for (int t = tid; t < YHX * YHY; t += YNT) {
      const int lx = t % YHX, ly = t / YHX;
      const int i = i0 - 1 + lx, j = j0 - 1 + ly;
      const bool in = (k >= 0) && (k < nz) && (i >= 0) && (i < nx) && (j >= 0) && (j < ny);
      const int64_t idx = in ? ((int64_t)k * ny + j) * nx + i : 0;
      sm.H[hs][0][ly][lx] = in ? a.Hin[idx] : T(0);
      sm.H[hs][1][ly][lx] = in ? a.Hin[nc + idx] : T(0);
      sm.H[hs][2][ly][lx] = in ? a.Hin[2 * nc + idx] : T(0);
      sm.M[ms][ly][lx] = in ? a.mat[idx] : ID(0);
    }
  };

  int sp = s_beg;
  load_plane(k0 - 1);
  for (int k = k0; k <= k1; ++k) {
    const bool live = k < nz;
    if (live) load_plane(k);
    if (tid == 0) {
      while (sp < s_end && a.src[sp].k < k) ++sp;
      int sq = sp;
      while (sq < s_end && a.src[sq].k == k) ++sq;
      sm.rng[0] = sp;
      sm.rng[1] = sq;
    }
    __syncthreads();  // (A) plane k staged
    const int r0 = sm.rng[0], r1 = sm.rng[1];
    const int es = k & 1, esp = (k + 1) & 1;
    const int hs = k % 3, hsp = (k + 2) % 3;
    // ---- E^{n+1}[k] on tile + high halo
    for (int t = tid; t < YEX * YEY; t += YNT) {
      const int lx = t % YEX, ly = t / YEX;
      const int i = i0 + lx, j = j0 + ly;
      T ex = T(0), ey = T(0), ez = T(0);
      if (live && i < nx && j < ny) {
        const int hx = lx + 1, hy = ly + 1;
        const int64_t idx = ((int64_t)k * ny + j) * nx + i;
        const T rxd = axv(a.ax, ntot, AX_RDD, i);
        const T ryd = axv(a.ax, ntot, AX_RDD, nx + j);
        const T rzd = axv(a.ax, ntot, AX_RDD, nx + ny + k);
        T ca, cb;
        // (curl H)_x = dHz/dy - dHy/dz
        e_coef_at(a, sm, 0, lx, ly, i, j, k, ca, cb);
        ex = ca * a.Ein[idx] + cb * ((sm.H[hs][2][hy][hx] - sm.H[hs][2][hy - 1][hx]) * ryd -
                                     (sm.H[hs][1][hy][hx] - sm.H[hsp][1][hy][hx]) * rzd);
        // (curl H)_y = dHx/dz - dHz/dx
        e_coef_at(a, sm, 1, lx, ly, i, j, k, ca, cb);
        ey = ca * a.Ein[nc + idx] + cb * ((sm.H[hs][0][hy][hx] - sm.H[hsp][0][hy][hx]) * rzd -
                                          (sm.H[hs][2][hy][hx] - sm.H[hs][2][hy][hx - 1]) * rxd);
        // (curl H)_z = dHy/dx - dHx/dy
        e_coef_at(a, sm, 2, lx, ly, i, j, k, ca, cb);
        ez = ca * a.Ein[2 * nc + idx] + cb * ((sm.H[hs][1][hy][hx] - sm.H[hs][1][hy][hx - 1]) * rxd -
                                              (sm.H[hs][0][hy][hx] - sm.H[hs][0][hy - 1][hx]) * ryd);
      }
      sm.E[es][0][ly][lx] = ex;
      sm.E[es][1][ly][lx] = ey;
      sm.E[es][2][ly][lx] = ez;
    }
    __syncthreads();  // (B)
    // ---- sources of plane k: E -= Cb w u   (B = -w V_e, divided by V_e)
    if (r1 > r0) {
      for (int s = r0 + tid; s < r1; s += YNT) {
        const PortEntry pe = a.src[s];
        const int i = i0 + pe.lx, j = j0 + pe.ly;
        if (i < nx && j < ny) {
          T ca, cb;
          e_coef_at(a, sm, pe.comp, pe.lx, pe.ly, i, j, k, ca, cb);
          atomicAdd(&sm.E[es][pe.comp][pe.ly][pe.lx], -cb * (T)pe.w * a.u[pe.port]);
        }
      }
      __syncthreads();  // (C)
    }
    const int i = i0 + tx, j = j0 + ty;
    const bool own = i < nx && j < ny;
    if (k < k1) {
      if (own) {
        const int64_t idx = ((int64_t)k * ny + j) * nx + i;
        a.Eout[idx] = sm.E[es][0][ty][tx];
        a.Eout[nc + idx] = sm.E[es][1][ty][tx];
        a.Eout[2 * nc + idx] = sm.E[es][2][ty][tx];
      }
      for (int s = p_beg + tid; s < p_end; s += YNT) {
        const PortEntry pe = a.prb[s];
        if (pe.k == k) atomicAdd(&a.y[pe.port], (T)pe.w * sm.E[es][pe.comp][pe.ly][pe.lx]);
      }
    }
    // ---- H^{n+3/2}[k-1] on the tile
    if (k > k0 && own) {
      const int kk = k - 1;
      const int64_t idx = ((int64_t)kk * ny + j) * nx + i;
      const int hx = tx + 1, hy = ty + 1;
      const T rdx = axv(a.ax, ntot, AX_RD, i);
      const T rdy = axv(a.ax, ntot, AX_RD, nx + j);
      const T rdz = axv(a.ax, ntot, AX_RD, nx + ny + kk);
      const T(*E0)[YEY][YEX] = sm.E[esp];  // E^{n+1}[kk]
      const T(*E1)[YEY][YEX] = sm.E[es];   // E^{n+1}[kk+1]
      T da[3], db[3];
      if (HOMOG_H) {
        da[0] = da[1] = da[2] = __ldg(a.ctab + 2 * a.nmat);
        db[0] = db[1] = db[2] = __ldg(a.ctab + 3 * a.nmat);
      } else {
        const int mk = kk & 3, mkm = (kk + 3) & 3;
        h_coef(a, sm.M[mk][hy][hx - 1], sm.M[mk][hy][hx], axv(a.ax, ntot, AX_WLO, i),
               axv(a.ax, ntot, AX_WHI, i), da[0], db[0]);
        h_coef(a, sm.M[mk][hy - 1][hx], sm.M[mk][hy][hx], axv(a.ax, ntot, AX_WLO, nx + j),
               axv(a.ax, ntot, AX_WHI, nx + j), da[1], db[1]);
        h_coef(a, sm.M[mkm][hy][hx], sm.M[mk][hy][hx], axv(a.ax, ntot, AX_WLO, nx + ny + kk),
               axv(a.ax, ntot, AX_WHI, nx + ny + kk), da[2], db[2]);
      }
      // mu dHx/dt = -(dEz/dy - dEy/dz)
      T hxv = da[0] * sm.H[hsp][0][hy][hx] -
              db[0] * ((E0[2][ty + 1][tx] - E0[2][ty][tx]) * rdy - (E1[1][ty][tx] - E0[1][ty][tx]) * rdz);
      // mu dHy/dt = -(dEx/dz - dEz/dx)
      T hyv = da[1] * sm.H[hsp][1][hy][hx] -
              db[1] * ((E1[0][ty][tx] - E0[0][ty][tx]) * rdz - (E0[2][ty][tx + 1] - E0[2][ty][tx]) * rdx);
      // mu dHz/dt = -(dEy/dx - dEx/dy)
      T hzv = da[2] * sm.H[hsp][2][hy][hx] -
              db[2] * ((E0[1][ty][tx + 1] - E0[1][ty][tx]) * rdx - (E0[0][ty + 1][tx] - E0[0][ty][tx]) * rdy);
      a.Hout[idx] = (i == 0) ? T(0) : hxv;        // normal H on the x walls
      a.Hout[nc + idx] = (j == 0) ? T(0) : hyv;
      a.Hout[2 * nc + idx] = (kk == 0) ? T(0) : hzv;
    }
  }
}

template <typename T, typename ID, bool HH>
static fdtd_status launch_yee_t(fdtd_grid *g, const void *u_row, void *y_row, int kchunk,
                                cudaStream_t s) {
  YeeArgs<T, ID> a;
  a.nx = g->nx; a.ny = g->ny; a.nz = g->nz; a.kchunk = kchunk; a.nc = g->nc;
  a.ntx = g->lists.ntx; a.nty = g->lists.nty;
  const T *in = g->fields[g->cur].as<T>();
  T *out = g->fields[g->cur ^ 1].as<T>();
  a.Ein = in; a.Hin = in + 3 * g->nc;
  a.Eout = out; a.Hout = out + 3 * g->nc;
  a.mat = g->mat.as<ID>();
  a.ax = g->axis.as<T>();
  a.mtab = g->mtab.as<T>();
  a.ctab = g->ctab.as<T>();
  a.nmat = g->nmat;
  a.inv_dt = (T)(1.0 / g->ctab_dt);
  a.src_ptr = g->lists.src_ptr.as<int32_t>();
  a.src = g->lists.src.as<PortEntry>();
  a.u = static_cast<const T *>(u_row);
  a.prb_ptr = g->lists.prb_ptr.as<int32_t>();
  a.prb = g->lists.prb.as<PortEntry>();
  a.y = static_cast<T *>(y_row);
  dim3 grid(g->lists.ntx, g->lists.nty, (g->nz + kchunk - 1) / kchunk);
  dim3 block(YTX, YTY);
  size_t smem = sizeof(YeeSmem<T, ID>);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(yee_fused_kernel<T, ID, HH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  yee_fused_kernel<T, ID, HH><<<grid, block, smem, s>>>(a);
  return after_launch("yee_fused_kernel");
}

static fdtd_status launch_yee(fdtd_grid *g, const void *u_row, void *y_row, int kchunk,
                              cudaStream_t s) {
  if (g->prec == FDTD_F64) {
    if (g->id_bytes == 1)
      return g->homog_h ? launch_yee_t<double, uint8_t, true>(g, u_row, y_row, kchunk, s)
                        : launch_yee_t<double, uint8_t, false>(g, u_row, y_row, kchunk, s);
    return g->homog_h ? launch_yee_t<double, uint16_t, true>(g, u_row, y_row, kchunk, s)
                      : launch_yee_t<double, uint16_t, false>(g, u_row, y_row, kchunk, s);
  }
  if (g->id_bytes == 1)
    return g->homog_h ? launch_yee_t<float, uint8_t, true>(g, u_row, y_row, kchunk, s)
                      : launch_yee_t<float, uint8_t, false>(g, u_row, y_row, kchunk, s);
  return g->homog_h ? launch_yee_t<float, uint16_t, true>(g, u_row, y_row, kchunk, s)
                    : launch_yee_t<float, uint16_t, false>(g, u_row, y_row, kchunk, s);
}

// z-chunk length: enough CTAs to fill every SM, with the last wave as full as
// possible (each chunk recomputes about two planes, so fewer chunks are
// preferred when the wave efficiency is equal).
int choose_kchunk(const fdtd_grid *g, int ntiles, int ctas_per_sm) {
  const int cap = 152 * ctas_per_sm;
  const int maxch = std::max(1, g->nz / 4);
  double best = -1;
  int best_k = g->nz;
  for (int nch = 1; nch <= maxch; ++nch) {
    const int kch = (g->nz + nch - 1) / nch;
    const int used = (g->nz + kch - 1) / kch;
    const long total = (long)ntiles * used;
    const long waves = (total + cap - 1) / cap;
    const double eff = (double)total / (double)(waves * cap) * (double)kch / (double)(kch + 2);
    if (eff > best + 1e-9) { best = eff; best_k = kch; }
  }
  return best_k;
}

// Leap-frog steps per captured graph (even, so a replay leaves cur unchanged).
constexpr int kGraphSteps = 32;

// The graph of kGraphSteps steps starting from parity g->cur, captured on a
// private stream the first time and whenever what it baked in has changed.
static fdtd_status step_graph(fdtd_grid *g, int kind, int kchunk, cudaStream_t s, cudaGraphExec_t *out,
                              int64_t *launches) {
  const int m = (int)g->ports.size(), p = (int)g->probes.size();
  if (m) FDTD_CHECK(g->u_graph.alloc((size_t)kGraphSteps * m * g->elem, s));
  if (p) FDTD_CHECK(g->y_graph.alloc((size_t)kGraphSteps * p * g->elem, s));
  double dt = g->ctab_dt;
  uint64_t dtbits;
  memcpy(&dtbits, &dt, sizeof(dt));
  const bool split = kind == FDTD_KERNEL_SPLIT || kind == FDTD_KERNEL_MARCH;
  uint64_t key[12] = {(uint64_t)kind,
                      (uint64_t)g->homog_h,
                      (uint64_t)kchunk,
                      dtbits,
                      (uint64_t)(uintptr_t)g->ctab.ptr ^ ((uint64_t)g->ctab_version << 40),  // tables built from it
                      (uint64_t)(uintptr_t)g->lists.src_ptr.ptr,
                      (uint64_t)(uintptr_t)g->lists.prb_ptr.ptr,
                      (uint64_t)(uintptr_t)g->emat.ptr ^ ((uint64_t)(uintptr_t)g->ecoef.ptr << 1),
                      (uint64_t)(uintptr_t)g->u_graph.ptr ^ ((uint64_t)(uintptr_t)g->y_graph.ptr << 1),
                      (uint64_t)g->lists.tx << 32 | (uint64_t)g->lists.ty,
                      (uint64_t)(split ? yee_split_vw(g) + 8 * yee_march_vw(g) + 64 * (int)yee_split_precoef(g) : 0) << 32 | (uint64_t)(split ? yee_split_lz(g) : 0) |
                          (uint64_t)(getenv("FDTDMOR_SLAB") ? atoi(getenv("FDTDMOR_SLAB")) : g->tune_slab) << 16,
                      (uint64_t)(uintptr_t)g->fields[0].ptr ^ ((uint64_t)(uintptr_t)g->fields[1].ptr << 1)};
  const int c = g->cur;
  if (g->ygraph[c] && memcmp(key, g->ygraph_key[c], sizeof(key)) == 0) {
    *out = g->ygraph[c];
    *launches = g->ygraph_launches[c];
    return FDTD_OK;
  }
  if (g->ygraph[c]) {
    cudaGraphExecDestroy(g->ygraph[c]);
    g->ygraph[c] = nullptr;
  }
  if (!g->cap_stream) FDTD_CHECK_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
  cudaStream_t cs = g->cap_stream;
  const int64_t launches_before = fdtd_launch_count(0);
  FDTD_CHECK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  fdtd_status st = FDTD_OK;
  if (p && cudaMemsetAsync(g->y_graph.ptr, 0, (size_t)kGraphSteps * p * g->elem, cs) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "graph memset");
  for (int n = 0; n < kGraphSteps && st == FDTD_OK; ++n) {
    const char *ur = m ? static_cast<const char *>(g->u_graph.ptr) + (size_t)n * m * g->elem : nullptr;
    char *yr = p ? static_cast<char *>(g->y_graph.ptr) + (size_t)n * p * g->elem : nullptr;
    if (kind == FDTD_KERNEL_SPLIT) st = launch_yee_split(g, ur, yr, cs);
    else if (kind == FDTD_KERNEL_MARCH) st = launch_yee_march(g, ur, yr, cs);
    else if (kind == FDTD_KERNEL_TMA) st = launch_yee_tma(g, ur, yr, kchunk, cs);
    else st = launch_yee(g, ur, yr, kchunk, cs);
    g->cur ^= 1;
  }
  g->cur = c;
  const int64_t captured = fdtd_launch_count(0) - launches_before;
  add_launches(-captured);  // captured, not launched
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &graph);
  if (st != FDTD_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "graph capture");
  const cudaError_t e2 = cudaGraphInstantiate(&g->ygraph[c], graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) {
    g->ygraph[c] = nullptr;
    return cuda_fail(e2, "graph instantiate");
  }
  memcpy(g->ygraph_key[c], key, sizeof(key));
  g->ygraph_launches[c] = captured;
  *out = g->ygraph[c];
  *launches = captured;
  return FDTD_OK;
}

fdtd_status yee_run(fdtd_grid *g, double dt, int64_t nsteps, const void *u, void *y,
                    int reset_fields, cudaStream_t s) {
  FDTD_REQUIRE(dt > 0, "dt must be > 0");
  FDTD_REQUIRE(nsteps >= 0, "nsteps must be >= 0");
  FDTD_REQUIRE(nsteps == 0 || g->ports.empty() || u, "u is required when the grid has sources");
  FDTD_REQUIRE(nsteps == 0 || g->probes.empty() || y, "y is required when the grid has probes");
  FDTD_CHECK(ensure_coef_table(g, dt, s));
  int kind = g->kernel;
  if (const char *e = getenv("FDTDMOR_YEE")) {  // override for measurements
    const std::string v(e);
    kind = v == "persist" ? FDTD_KERNEL_PERSIST : v == "split" ? FDTD_KERNEL_SPLIT
         : v == "tma" ? FDTD_KERNEL_TMA : v == "fused" ? FDTD_KERNEL_FUSED
         : v == "march" ? FDTD_KERNEL_MARCH : kind;
  }
  if (kind == FDTD_KERNEL_TMA && !yee_tma_eligible(g)) kind = FDTD_KERNEL_FUSED;
  // AUTO: the fused one-pass form where its 128-cell FP32 tiles fill the grid
  // and there are enough of them to fill the GPU, else the split pair
  if (kind == FDTD_KERNEL_AUTO)
    kind = (yee_march_vw(g) == 4 && g->nc >= ((int64_t)1 << 22)) ? FDTD_KERNEL_MARCH : FDTD_KERNEL_SPLIT;
  int ttx = YTX, tty = YTY;
  if (kind == FDTD_KERNEL_TMA) yee_tma_tile(&ttx, &tty);
  if (kind == FDTD_KERNEL_PERSIST || kind == FDTD_KERNEL_SPLIT) ttx = 32 * yee_split_vw(g);
  if (kind == FDTD_KERNEL_MARCH) ttx = 32 * yee_march_vw(g);
  FDTD_CHECK(build_tile_lists(g, ttx, tty, s));
  if (reset_fields) {
    FDTD_CHECK_CUDA(cudaMemsetAsync(g->fields[g->cur].ptr, 0, (size_t)6 * g->nc * g->elem, s));
  }
  const int m = (int)g->ports.size(), p = (int)g->probes.size();
  if (p && nsteps) FDTD_CHECK_CUDA(cudaMemsetAsync(y, 0, (size_t)nsteps * p * g->elem, s));
  if (kind == FDTD_KERNEL_PERSIST) return run_yee_stream(g, nsteps, u, y, s);
  const int kchunk = choose_kchunk(g, g->lists.ntx * g->lists.nty, kind == FDTD_KERNEL_TMA ? 3 : 4);
  auto one_step = [&](const void *ur, void *yr) -> fdtd_status {
    if (kind == FDTD_KERNEL_SPLIT) return launch_yee_split(g, ur, yr, s);
    if (kind == FDTD_KERNEL_MARCH) return launch_yee_march(g, ur, yr, s);
    if (kind == FDTD_KERNEL_TMA) return launch_yee_tma(g, ur, yr, kchunk, s);
    return launch_yee(g, ur, yr, kchunk, s);
  };
  int64_t n = 0;
  if (nsteps > 2 * kGraphSteps && !graphs_off()) {
    // one direct step first (lazily built device tables are made outside any
    // capture), then whole chunks as replays of a captured graph: u rows are
    // staged into a fixed buffer before each replay and y rows copied out
    FDTD_CHECK(one_step(u, y));
    g->cur ^= 1;
    n = 1;
    cudaGraphExec_t exec = nullptr;
    int64_t per_replay = 0;
    FDTD_CHECK(step_graph(g, kind, kchunk, s, &exec, &per_replay));
    for (; n + kGraphSteps <= nsteps; n += kGraphSteps) {
      if (m) FDTD_CHECK_CUDA(cudaMemcpyAsync(g->u_graph.ptr, static_cast<const char *>(u) + (size_t)n * m * g->elem,
                                             (size_t)kGraphSteps * m * g->elem, cudaMemcpyDeviceToDevice, s));
      FDTD_CHECK_CUDA(cudaGraphLaunch(exec, s));
      add_launches(per_replay);
      if (p) FDTD_CHECK_CUDA(cudaMemcpyAsync(static_cast<char *>(y) + (size_t)n * p * g->elem, g->y_graph.ptr,
                                             (size_t)kGraphSteps * p * g->elem, cudaMemcpyDeviceToDevice, s));
    }
  }
  for (; n < nsteps; ++n) {
    const char *ur = u ? static_cast<const char *>(u) + (size_t)n * m * g->elem : nullptr;
    char *yr = y ? static_cast<char *>(y) + (size_t)n * p * g->elem : nullptr;
    FDTD_CHECK(one_step(ur, yr));
    g->cur ^= 1;
  }
  return FDTD_OK;
}

}  // namespace fdtdmor

using namespace fdtdmor;

extern "C" {

fdtd_status fdtd_grid_set_kernel(fdtd_grid *g, int kernel) {
  FDTD_REQUIRE(g, "fdtd_grid_set_kernel: NULL grid");
  FDTD_REQUIRE(kernel >= FDTD_KERNEL_AUTO && kernel <= FDTD_KERNEL_MARCH, "fdtd_grid_set_kernel: unknown kernel %d",
               kernel);
  FDTD_REQUIRE(kernel != FDTD_KERNEL_TMA || yee_tma_eligible(g),
               "fdtd_grid_set_kernel: the TMA form needs nx a multiple of %d", g->id_bytes == 1 ? 16 : 8);
  g->kernel = kernel;
  return FDTD_OK;
}

fdtd_status fdtd_grid_autotune(fdtd_grid *g, double dt, int trial_steps, int *vw_out, int *lz_out,
                               fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(g, "fdtd_grid_autotune: NULL grid");
  FDTD_REQUIRE(dt > 0 && trial_steps >= 1, "fdtd_grid_autotune: need dt > 0 and trial_steps >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t fbytes = (size_t)6 * g->nc * g->elem;
  const int m = (int)g->ports.size(), p = (int)g->probes.size();
  DevBuf save, ub, yb;
  struct Rel {
    DevBuf *a, *b, *c;
    cudaStream_t s;
    ~Rel() { a->release(s); b->release(s); c->release(s); }
  } rel{&save, &ub, &yb, s};
  FDTD_CHECK(save.alloc(fbytes, s));
  if (m) FDTD_CHECK(ub.alloc((size_t)trial_steps * m * g->elem, s));
  if (p) FDTD_CHECK(yb.alloc((size_t)trial_steps * p * g->elem, s));
  if (m) FDTD_CHECK_CUDA(cudaMemsetAsync(ub.ptr, 0, (size_t)trial_steps * m * g->elem, s));
  FDTD_CHECK_CUDA(cudaMemcpyAsync(save.ptr, g->fields[g->cur].ptr, fbytes, cudaMemcpyDeviceToDevice, s));
  const int cur0 = g->cur, kind0 = g->kernel;
  g->kernel = FDTD_KERNEL_SPLIT;
  cudaEvent_t e0, e1;
  FDTD_CHECK_CUDA(cudaEventCreate(&e0));
  FDTD_CHECK_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bvw = 1, blz = 1;
  fdtd_status st = FDTD_OK;
  for (int vw = 1; vw <= 16 / g->elem && st == FDTD_OK; vw *= 2) {
    if (g->nx % vw) continue;
    for (int lz = 1; lz <= 8 && lz <= std::max(1, g->nz) && st == FDTD_OK; lz *= 2) {
      g->tune_vw = vw;
      g->tune_lz = lz;
      st = yee_run(g, dt, std::min(trial_steps, 4), ub.ptr, yb.ptr, 0, s);  // warm-up, lists, graphs
      if (st != FDTD_OK) break;
      cudaEventRecord(e0, s);
      st = yee_run(g, dt, trial_steps, ub.ptr, yb.ptr, 0, s);
      cudaEventRecord(e1, s);
      if (st != FDTD_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) { st = cuda_fail(cudaGetLastError(), "autotune"); break; }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; bvw = vw; blz = lz; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g->kernel = kind0;
  g->tune_vw = bvw;
  g->tune_lz = blz;
  g->cur = cur0;
  FDTD_CHECK(st);
  FDTD_CHECK_CUDA(cudaMemcpyAsync(g->fields[g->cur].ptr, save.ptr, fbytes, cudaMemcpyDeviceToDevice, s));
  if (vw_out) *vw_out = bvw;
  if (lz_out) *lz_out = blz;
  return FDTD_OK;
}

fdtd_status fdtd_step(fdtd_grid *g, double dt, int64_t nsteps, const void *u, void *y,
                      int reset_fields, fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(g, "fdtd_step: NULL grid");
  cudaStream_t s = (cudaStream_t)stream;
  FDTD_CHECK(watchdog_before(g, u, reset_fields, s));
  FDTD_CHECK(yee_run(g, dt, nsteps, u, y, reset_fields, s));
  return watchdog_after(g, u, reset_fields, s);
}

fdtd_status fdtd_step_host(fdtd_grid *g, double dt, int64_t nsteps, const void *u_host,
                           void *y_host, int reset_fields, fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(g, "fdtd_step_host: NULL grid");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ub = (size_t)nsteps * g->ports.size() * g->elem;
  const size_t yb = (size_t)nsteps * g->probes.size() * g->elem;
  FDTD_REQUIRE(ub == 0 || u_host, "u_host is required when the grid has sources");
  FDTD_REQUIRE(yb == 0 || y_host, "y_host is required when the grid has probes");
  if (ub) {
    FDTD_CHECK(g->u_stage.alloc(ub, s));
    FDTD_CHECK_CUDA(cudaMemcpyAsync(g->u_stage.ptr, u_host, ub, cudaMemcpyHostToDevice, s));
  }
  if (yb) FDTD_CHECK(g->y_stage.alloc(yb, s));
  FDTD_CHECK(watchdog_before(g, u_host, reset_fields, s));
  FDTD_CHECK(yee_run(g, dt, nsteps, ub ? g->u_stage.ptr : nullptr, yb ? g->y_stage.ptr : nullptr,
                     reset_fields, s));
  if (yb) FDTD_CHECK_CUDA(cudaMemcpyAsync(y_host, g->y_stage.ptr, yb, cudaMemcpyDeviceToHost, s));
  FDTD_CHECK(watchdog_after(g, u_host, reset_fields, s));
  FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  return FDTD_OK;
}

}  // extern "C"
