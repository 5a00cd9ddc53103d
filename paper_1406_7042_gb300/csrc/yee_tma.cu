// A2 (fast path): the fused Yee leap-frog of Eq. (matrix) with TMA-fed plane
// pipelining, for grids whose rows are 16-byte aligned (nx a multiple of 16
// with uint8 ids / 8 with uint16 ids).
//
// Each CTA owns a 32 x 7 xy tile and marches a chunk of z planes with 32 x 8
// threads: thread (tx, ty) computes E^{n+1} at (tx, ty) of the 33 x 8 region
// (tile plus its +y halo row); the 8 threads of the halo row that have no H
// cell also compute the +x halo column.  Per plane the CTA needs H^{n+1/2} and
// the cell ids with a one-cell halo: one elected thread issues
// cp.async.bulk.tensor loads of these boxes S-4 planes ahead into an S-stage
// shared-memory ring (with E^n on the region), each stage completed through
// its own mbarrier.  Boxes start on 16-byte boundaries (x rounded down, the extra
// columns are padding) and coordinates outside the grid read as zero, which is
// also the PEC value of tangential E and normal H on the walls.
//
// H^{n+3/2} lags E^{n+1} by two planes (iteration k computes E[k], stores
// E[k-1] and computes H[k-2] from E[k-2], E[k-1]), so nothing computed in an
// iteration is read in the same iteration and one barrier per plane suffices
// (one more on the rare planes that carry sources).  Where every cell a tile
// sees at a plane has one material (flag from tile_uniform_kernel) the
// per-edge averaging is skipped.
#include <cuda.h>

#include <algorithm>
#include <cstdlib>

#include "common.cuh"
#include "grid_internal.cuh"
#include "yee_internal.cuh"
#include "tma_util.cuh"

namespace fdtdmor {

constexpr int QTX = 32, QTY = 7;              // tile of cells
constexpr int QBX = 32, QBY = 8, QNT = QBX * QBY;  // threads: the 33 x 8 E region minus its x-halo column
constexpr int QEX = QTX + 1, QEY = QTY + 1;     // E^{n+1} region: tile + high halo
constexpr int QSLOTS = 3;                       // E^{n+1} planes kept in shared memory

template <typename T, typename ID>
struct QLayout {
  static constexpr int HX = QTX + 8, HY = QTY + 2;    // H box from (i0-4, j0-1)
  static constexpr int EX = QTX + 4, EY = QTY + 1;    // E box from (i0, j0)
  static constexpr int MPAD = 16 / (int)sizeof(ID);   // id box from (i0-MPAD, j0-1)
  static constexpr int MX = QTX + 2 * MPAD, MY = QTY + 2;
  static constexpr int rup(int b) { return (b + 127) / 128 * 128; }
  static constexpr int HB = rup(HX * HY * (int)sizeof(T));
  static constexpr int EB = rup(EX * EY * (int)sizeof(T));
  static constexpr int MB_ = rup(MX * MY * (int)sizeof(ID));
  static constexpr int STAGE = 3 * HB + 3 * EB + MB_;
  static constexpr uint32_t TX_BYTES = 3u * HX * HY * sizeof(T) + 3u * EX * EY * sizeof(T) + MX * MY * sizeof(ID);
};

struct QMaps {
  CUtensorMap E[2][3];
  CUtensorMap H[2][3];
  CUtensorMap M;
};

// Material of every cell an E or H coefficient of tile t at plane k can see
// (x in [i0-1, i0+32], y in [j0-1, j0+7], z in {k-1, k}), or -1 if they differ.
template <typename ID>
__global__ void tile_uniform_kernel(const ID *__restrict__ mat, int nx, int ny, int nz, int ntx, int nty,
                                    int *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int ntiles = ntx * nty;
  if (t >= ntiles * nz) return;
  const int k = t / ntiles, tile = t % ntiles;
  const int i0 = (tile % ntx) * QTX, j0 = (tile / ntx) * QTY;
  int m0 = -2;
  bool uni = true;
  for (int kk = max(0, k - 1); kk <= k && uni; ++kk)
    for (int j = max(0, j0 - 1); j <= min(ny - 1, j0 + QTY) && uni; ++j)
      for (int i = max(0, i0 - 1); i <= min(nx - 1, i0 + QTX); ++i) {
        const int m = mat[((int64_t)kk * ny + j) * nx + i];
        if (m0 == -2) m0 = m;
        else if (m != m0) { uni = false; break; }
      }
  out[t] = uni ? m0 : -1;
}

template <typename T, typename ID, bool HOMOG_H, int S>
__global__ void __launch_bounds__(QNT, sizeof(T) == 4 ? 3 : 1) yee_tma_kernel(const __grid_constant__ QMaps maps, YeeArgs<T, ID> a,
                                                      int src_buf, const int *__restrict__ uflag, unsigned *err) {
  using Lay = QLayout<T, ID>;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *ring = smem;
  T(*En)[3][QEY][QEX] = reinterpret_cast<T(*)[3][QEY][QEX]>(smem + S * Lay::STAGE);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S * Lay::STAGE + QSLOTS * 3 * QEY * QEX * sizeof(T));
  int *rng = reinterpret_cast<int *>(bars + S);   // [2][2]: source range of planes k (k & 1)

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * QBX + tx;
  const int i0 = blockIdx.x * QTX, j0 = blockIdx.y * QTY;
  const int k0 = blockIdx.z * a.kchunk;
  if (k0 >= a.nz) return;
  const int k1 = min(a.nz, k0 + a.kchunk);
  const int nx = a.nx, ny = a.ny, nz = a.nz, ntot = nx + ny + nz;
  const int64_t nc = a.nc;
  const int tile = blockIdx.y * gridDim.x + blockIdx.x, ntiles = gridDim.x * gridDim.y;
  const int s_end = a.src_ptr[tile + 1];
  const int p_beg = a.prb_ptr[tile], p_end = a.prb_ptr[tile + 1];

  // planes p = k0-1 .. kmax are loaded; relative index r = p - (k0-1)
  const int kmax = min(k1, nz - 1);
  const int rmax = kmax - (k0 - 1);
  auto Hs = [&](int r, int c) { return reinterpret_cast<const T *>(ring + (r % S) * Lay::STAGE + c * Lay::HB); };
  // stage layout: H0 H1 H2 | E0 E1 E2 | ids
  auto Hst = [&](const unsigned char *st, int c) { return reinterpret_cast<const T *>(st + c * Lay::HB); };
  auto Est = [&](const unsigned char *st, int c) { return reinterpret_cast<const T *>(st + 3 * Lay::HB + c * Lay::EB); };
  auto Mst = [&](const unsigned char *st) { return reinterpret_cast<const ID *>(st + 3 * Lay::HB + 3 * Lay::EB); };
  auto issue = [&](int r) {
    unsigned char *st = ring + (r % S) * Lay::STAGE;
    uint64_t *bar = &bars[r % S];
    const int z = k0 - 1 + r;
    mbar_expect_tx(bar, Lay::TX_BYTES);
    for (int c = 0; c < 3; ++c) tma_load_3d(st + c * Lay::HB, &maps.H[src_buf][c], i0 - 4, j0 - 1, z, bar);
    for (int c = 0; c < 3; ++c) tma_load_3d(st + 3 * Lay::HB + c * Lay::EB, &maps.E[src_buf][c], i0, j0, z, bar);
    tma_load_3d(st + 3 * Lay::HB + 3 * Lay::EB, &maps.M, i0 - Lay::MPAD, j0 - 1, z, bar);
  };

  if (tid == 0) {
    for (int q = 0; q < S; ++q) mbar_init(&bars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int r = 0; r <= min(S - 4, rmax); ++r) issue(r);
  }
  __syncthreads();

  // this thread's E positions: (tx, ty) of the 33 x 8 region and, for the
  // threads of the halo row, one cell of the x-halo column
  auto ax = [&](int table, int idx) { return __ldg(a.ax + table * ntot + idx); };
  const int ti = i0 + tx, tj = j0 + ty;
  const bool tile_row = ty < QTY;                   // owns an H cell and an E store
  const bool xhalo = (ty == QTY) && (tx < QEY);     // also computes E at (32, tx)
  const int cin = min(ti, nx - 1), cjn = min(tj, ny - 1);
  const T rxd = ax(AX_RDD, cin), ryd = ax(AX_RDD, nx + cjn), rdx = ax(AX_RD, cin), rdy = ax(AX_RD, nx + cjn);
  const T wxl = ax(AX_WLO, cin), wxh = ax(AX_WHI, cin), wyl = ax(AX_WLO, nx + cjn), wyh = ax(AX_WHI, nx + cjn);
  const int hi_i = min(i0 + QTX, nx - 1), hi_j = min(j0 + tx, ny - 1);  // x-halo cell (i0+32, j0+tx)
  const T hrxd = ax(AX_RDD, hi_i), hryd = ax(AX_RDD, nx + hi_j);
  const T hwxl = ax(AX_WLO, hi_i), hwxh = ax(AX_WHI, hi_i), hwyl = ax(AX_WLO, nx + hi_j), hwyh = ax(AX_WHI, nx + hi_j);

  // E^{n+1} at region position (lx, ly), global (i, j), plane k (relative r)
  auto e_at = [&](int lx, int ly, int i, int j, int k, const unsigned char *sk, const unsigned char *skm, int uni,
                  T rxd_, T ryd_, T wxl_, T wxh_, T wyl_, T wyh_, T rzd, T wzl, T wzh, T &ex, T &ey, T &ez) {
    const T *H0 = Hst(sk, 0), *H1 = Hst(sk, 1), *H2 = Hst(sk, 2), *Hm0 = Hst(skm, 0), *Hm1 = Hst(skm, 1);
    const int hI = (ly + 1) * Lay::HX + lx + 4, eI = ly * Lay::EX + lx;
    const T eo[3] = {Est(sk, 0)[eI], Est(sk, 1)[eI], Est(sk, 2)[eI]};
    T cax, cbx, cay, cby, caz, cbz;
    if (uni >= 0) {
      const T ca = __ldg(a.ctab + uni), cb = __ldg(a.ctab + a.nmat + uni);
      cax = cay = caz = ca;
      cbx = cby = cbz = cb;
    } else {
      const ID *Mk = Mst(sk), *Mm = Mst(skm);
      const int mI = (ly + 1) * Lay::MX + lx + Lay::MPAD;
      e_coef(a, Mm[mI - Lay::MX], Mm[mI], Mk[mI - Lay::MX], Mk[mI], wyl_, wyh_, wzl, wzh, cax, cbx);
      e_coef(a, Mm[mI - 1], Mm[mI], Mk[mI - 1], Mk[mI], wxl_, wxh_, wzl, wzh, cay, cby);
      e_coef(a, Mk[mI - Lay::MX - 1], Mk[mI - Lay::MX], Mk[mI - 1], Mk[mI], wxl_, wxh_, wyl_, wyh_, caz, cbz);
    }
    if (j == 0 || k == 0) cax = cbx = T(0);
    if (i == 0 || k == 0) cay = cby = T(0);
    if (i == 0 || j == 0) caz = cbz = T(0);
    ex = cax * eo[0] + cbx * ((H2[hI] - H2[hI - Lay::HX]) * ryd_ - (H1[hI] - Hm1[hI]) * rzd);
    ey = cay * eo[1] + cby * ((H0[hI] - Hm0[hI]) * rzd - (H2[hI] - H2[hI - 1]) * rxd_);
    ez = caz * eo[2] + cbz * ((H1[hI] - H1[hI - 1]) * rxd_ - (H0[hI] - H0[hI - Lay::HX]) * ryd_);
  };
  const bool own_e = ti < nx && tj < ny;
  const bool own_h = xhalo && i0 + QTX < nx && j0 + tx < ny;

  int sp = a.src_ptr[tile];
  // source range of plane k goes to rng[2*(k&1)..]; written one plane ahead by
  // thread 0 and published by the end-of-plane barrier
  auto src_range = [&](int k) {
    while (sp < s_end && a.src[sp].k < k) ++sp;
    int sq = sp;
    while (sq < s_end && a.src[sq].k == k) ++sq;
    rng[2 * (k & 1)] = sp;
    rng[2 * (k & 1) + 1] = sq;
  };
  if (tid == 0) src_range(k0);
  __syncthreads();
  bool ok = mbar_wait(&bars[0], 0);
  int waited = 0;
  for (int k = k0; k <= k1 + 1; ++k) {
    const int r = k - k0 + 1;
    const bool e_live = k <= kmax;        // E^{n+1}[k] computed from loaded data
    if (tid == 0) {
      if (r + S - 4 <= rmax && r >= 1) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(r + S - 4);
      }
      src_range(k + 1);
    }
    if (e_live) {
      if (!mbar_wait(&bars[r % S], (r / S) & 1)) ok = false;
      waited = r;
    }
    const unsigned char *sk = ring + (r % S) * Lay::STAGE;                // plane k
    const unsigned char *skm = ring + ((r + S - 1) % S) * Lay::STAGE;     // plane k-1
    const unsigned char *sk2 = ring + ((r + S - 2) % S) * Lay::STAGE;     // plane k-2
    const unsigned char *sk3 = ring + ((r + S - 3) % S) * Lay::STAGE;     // plane k-3
    const int es = k % QSLOTS, es1 = (k + QSLOTS - 1) % QSLOTS, es2 = (k + QSLOTS - 2) % QSLOTS;
    // ---- E^{n+1}[k] on tile + halo (zero beyond the top wall)
    if (k <= k1) {
      T ex = 0, ey = 0, ez = 0;
      T hx = 0, hy = 0, hz = 0;
      if (e_live && ok) {
        const int uni = __ldg(uflag + (int64_t)k * ntiles + tile);
        const T rzd = ax(AX_RDD, nx + ny + k), wzl = ax(AX_WLO, nx + ny + k), wzh = ax(AX_WHI, nx + ny + k);
        if (own_e) e_at(tx, ty, ti, tj, k, sk, skm, uni, rxd, ryd, wxl, wxh, wyl, wyh, rzd, wzl, wzh, ex, ey, ez);
        if (own_h)
          e_at(QTX, tx, i0 + QTX, j0 + tx, k, sk, skm, uni, hrxd, hryd, hwxl, hwxh, hwyl, hwyh, rzd, wzl, wzh, hx, hy, hz);
      }
      En[es][0][ty][tx] = ex; En[es][1][ty][tx] = ey; En[es][2][ty][tx] = ez;
      if (xhalo) { En[es][0][tx][QTX] = hx; En[es][1][tx][QTX] = hy; En[es][2][tx][QTX] = hz; }
    }
    // ---- sources of plane k (rare): E -= Cb w u, after the plane is complete
    const int r0 = rng[2 * (k & 1)], r1 = e_live ? rng[2 * (k & 1) + 1] : r0;
    if (r1 > r0) {
      __syncthreads();
      for (int q = r0 + tid; q < r1; q += QNT) {
        const PortEntry pe = a.src[q];
        const int i = i0 + pe.lx, j = j0 + pe.ly;
        if (i < nx && j < ny && pe.ly <= QTY) {
          const int uni = __ldg(uflag + (int64_t)k * ntiles + tile);
          const T wzl = ax(AX_WLO, nx + ny + k), wzh = ax(AX_WHI, nx + ny + k);
          T ca, cb;
          if (uni >= 0) cb = __ldg(a.ctab + a.nmat + uni);
          else {
            const ID *Mk = Mst(sk), *Mm = Mst(skm);
            const int mI = (pe.ly + 1) * Lay::MX + pe.lx + Lay::MPAD;
            const T wxl_ = ax(AX_WLO, i), wxh_ = ax(AX_WHI, i), wyl_ = ax(AX_WLO, nx + j), wyh_ = ax(AX_WHI, nx + j);
            if (pe.comp == 0) e_coef(a, Mm[mI - Lay::MX], Mm[mI], Mk[mI - Lay::MX], Mk[mI], wyl_, wyh_, wzl, wzh, ca, cb);
            else if (pe.comp == 1) e_coef(a, Mm[mI - 1], Mm[mI], Mk[mI - 1], Mk[mI], wxl_, wxh_, wzl, wzh, ca, cb);
            else e_coef(a, Mk[mI - Lay::MX - 1], Mk[mI - Lay::MX], Mk[mI - 1], Mk[mI], wxl_, wxh_, wyl_, wyh_, ca, cb);
          }
          if ((pe.comp == 0 && (j == 0 || k == 0)) || (pe.comp == 1 && (i == 0 || k == 0)) ||
              (pe.comp == 2 && (i == 0 || j == 0)))
            cb = T(0);
          atomicAdd(&En[es][pe.comp][pe.ly][pe.lx], -cb * (T)pe.w * a.u[pe.port]);
        }
      }
    }
    const bool own = tile_row && ti < nx && tj < ny;
    // ---- E^{n+1}[k-1] (complete since the last barrier) to global, probes
    const int ke = k - 1;
    if (ke >= k0 && ke < k1) {
      if (own) {
        const int64_t idx = ((int64_t)ke * ny + tj) * nx + ti;
        a.Eout[idx] = En[es1][0][ty][tx];
        a.Eout[nc + idx] = En[es1][1][ty][tx];
        a.Eout[2 * nc + idx] = En[es1][2][ty][tx];
      }
      for (int q = p_beg + tid; q < p_end; q += QNT) {
        const PortEntry pe = a.prb[q];
        if (pe.k == ke) atomicAdd(&a.y[pe.port], (T)pe.w * En[es1][pe.comp][pe.ly][pe.lx]);
      }
    }
    // ---- H^{n+3/2}[k-2] from E^{n+1}[k-2], E^{n+1}[k-1]
    const int kk = k - 2;
    if (kk >= k0 && kk < k1 && own && ok) {
      const int64_t idx = ((int64_t)kk * ny + tj) * nx + ti;
      const T rdz = ax(AX_RD, nx + ny + kk);
      const int hI = (ty + 1) * Lay::HX + tx + 4;
      const T(*E0)[QEY][QEX] = En[es2];  // E^{n+1}[kk]
      const T(*E1)[QEY][QEX] = En[es1];  // E^{n+1}[kk+1]
      T da[3], db[3];
      if (HOMOG_H) {
        da[0] = da[1] = da[2] = __ldg(a.ctab + 2 * a.nmat);
        db[0] = db[1] = db[2] = __ldg(a.ctab + 3 * a.nmat);
      } else {
        const int uni = __ldg(uflag + (int64_t)kk * ntiles + tile);
        if (uni >= 0) {
          da[0] = da[1] = da[2] = __ldg(a.ctab + 2 * a.nmat + uni);
          db[0] = db[1] = db[2] = __ldg(a.ctab + 3 * a.nmat + uni);
        } else {
          const ID *Mc = Mst(sk2), *Mb = Mst(sk3);
          const int mI = (ty + 1) * Lay::MX + tx + Lay::MPAD;
          h_coef(a, Mc[mI - 1], Mc[mI], wxl, wxh, da[0], db[0]);
          h_coef(a, Mc[mI - Lay::MX], Mc[mI], wyl, wyh, da[1], db[1]);
          h_coef(a, Mb[mI], Mc[mI], ax(AX_WLO, nx + ny + kk), ax(AX_WHI, nx + ny + kk), da[2], db[2]);
        }
      }
      const T *Ho0 = Hst(sk2, 0), *Ho1 = Hst(sk2, 1), *Ho2 = Hst(sk2, 2);
      const T hxv = da[0] * Ho0[hI] -
                    db[0] * ((E0[2][ty + 1][tx] - E0[2][ty][tx]) * rdy - (E1[1][ty][tx] - E0[1][ty][tx]) * rdz);
      const T hyv = da[1] * Ho1[hI] -
                    db[1] * ((E1[0][ty][tx] - E0[0][ty][tx]) * rdz - (E0[2][ty][tx + 1] - E0[2][ty][tx]) * rdx);
      const T hzv = da[2] * Ho2[hI] -
                    db[2] * ((E0[1][ty][tx + 1] - E0[1][ty][tx]) * rdx - (E0[0][ty + 1][tx] - E0[0][ty][tx]) * rdy);
      a.Hout[idx] = (ti == 0) ? T(0) : hxv;
      a.Hout[nc + idx] = (tj == 0) ? T(0) : hyv;
      a.Hout[2 * nc + idx] = (kk == 0) ? T(0) : hzv;
    }
    if (__syncthreads_or(!ok)) break;  // one barrier per plane
  }
  if (!ok) {
    // a wait gave up: record it, then let the copies this CTA issued land
    // (bounded) before the CTA exits and its shared memory is reused
    if (tid == 0) {
      atomicExch(err, 1u);
      const int last = min(rmax, waited + S - 4);
      for (int r = waited + 1; r <= last; ++r) mbar_wait(&bars[r % S], (r / S) & 1);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ host
void yee_tma_tile(int *tx, int *ty) {
  *tx = QTX;
  *ty = QTY;
}

bool yee_tma_eligible(const fdtd_grid *g) {
  if (getenv("FDTDMOR_NO_TMA")) return false;
  const int need = g->id_bytes == 1 ? 16 : 8;   // id rows 16-byte aligned (field rows follow)
  return g->nx % need == 0 && encode_fn() != nullptr;
}

// Tensor maps of the last grid used, with everything they encode: a later
// grid may reuse the same device addresses with other sizes or types.
struct TmaCache {
  QMaps maps;
  const void *f0 = nullptr, *f1 = nullptr, *mat = nullptr;
  int nx = 0, ny = 0, nz = 0, elem = 0, id_bytes = 0;
  bool same(const fdtd_grid *g) const {
    return f0 == g->fields[0].ptr && f1 == g->fields[1].ptr && mat == g->mat.ptr && nx == g->nx && ny == g->ny &&
           nz == g->nz && elem == g->elem && id_bytes == g->id_bytes;
  }
  void set(const fdtd_grid *g) {
    f0 = g->fields[0].ptr; f1 = g->fields[1].ptr; mat = g->mat.ptr;
    nx = g->nx; ny = g->ny; nz = g->nz; elem = g->elem; id_bytes = g->id_bytes;
  }
};

template <typename T, typename ID, bool HH>
static fdtd_status launch_tma_t(fdtd_grid *g, const void *u_row, void *y_row, int kchunk, cudaStream_t s,
                                QMaps &maps, unsigned *err) {
  constexpr int S = sizeof(T) == 4 ? 7 : 5;
  using Lay = QLayout<T, ID>;
  YeeArgs<T, ID> a;
  a.nx = g->nx; a.ny = g->ny; a.nz = g->nz; a.kchunk = kchunk; a.nc = g->nc;
  a.ntx = g->lists.ntx; a.nty = g->lists.nty;
  T *out = g->fields[g->cur ^ 1].as<T>();
  a.Ein = nullptr; a.Hin = nullptr;
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
  const size_t smem = (size_t)S * Lay::STAGE + QSLOTS * 3 * QEY * QEX * sizeof(T) + S * sizeof(uint64_t) + 4 * sizeof(int);
  static bool attr = false;
  if (!attr) {
    FDTD_CHECK_CUDA(cudaFuncSetAttribute(yee_tma_kernel<T, ID, HH, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    attr = true;
  }
  dim3 grid(g->lists.ntx, g->lists.nty, (g->nz + kchunk - 1) / kchunk);
  yee_tma_kernel<T, ID, HH, S><<<grid, dim3(QBX, QBY), smem, s>>>(maps, a, g->cur, g->uflag.as<int>(), err);
  return after_launch("yee_tma_kernel");
}

fdtd_status launch_yee_tma(fdtd_grid *g, const void *u_row, void *y_row, int kchunk, cudaStream_t s) {
  static thread_local TmaCache cache;  // tensor maps of the last grid (rebuilt when its buffers change)
  const bool f64 = g->prec == FDTD_F64;
  if (!cache.same(g)) {
    const CUtensorMapDataType ft = f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const int el = g->elem;
    for (int b = 0; b < 2; ++b) {
      char *base = (char *)g->fields[b].ptr;
      for (int c = 0; c < 3; ++c) {
        FDTD_CHECK(make_map(&cache.maps.E[b][c], ft, el, base + (size_t)c * g->nc * el, g, QTX + 4, QTY + 1));
        FDTD_CHECK(make_map(&cache.maps.H[b][c], ft, el, base + (size_t)(3 + c) * g->nc * el, g, QTX + 8, QTY + 2));
      }
    }
    if (g->id_bytes == 1)
      FDTD_CHECK(make_map(&cache.maps.M, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, g->mat.ptr, g, QTX + 32, QTY + 2));
    else
      FDTD_CHECK(make_map(&cache.maps.M, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, g->mat.ptr, g, QTX + 16, QTY + 2));
    cache.set(g);
  }
  unsigned *err = g->errflag.as<unsigned>();
  if (!g->uflag_ready) {
    const int n = g->lists.ntx * g->lists.nty * g->nz;
    FDTD_CHECK(g->uflag.alloc(sizeof(int) * std::max(1, n), s));
    if (g->id_bytes == 1)
      tile_uniform_kernel<uint8_t><<<(n + 255) / 256, 256, 0, s>>>(g->mat.as<uint8_t>(), g->nx, g->ny, g->nz,
                                                                  g->lists.ntx, g->lists.nty, g->uflag.as<int>());
    else
      tile_uniform_kernel<uint16_t><<<(n + 255) / 256, 256, 0, s>>>(g->mat.as<uint16_t>(), g->nx, g->ny, g->nz,
                                                                   g->lists.ntx, g->lists.nty, g->uflag.as<int>());
    FDTD_CHECK(after_launch("tile_uniform_kernel"));
    g->uflag_ready = true;
  }
  if (f64) {
    if (g->id_bytes == 1)
      return g->homog_h ? launch_tma_t<double, uint8_t, true>(g, u_row, y_row, kchunk, s, cache.maps, err)
                        : launch_tma_t<double, uint8_t, false>(g, u_row, y_row, kchunk, s, cache.maps, err);
    return g->homog_h ? launch_tma_t<double, uint16_t, true>(g, u_row, y_row, kchunk, s, cache.maps, err)
                      : launch_tma_t<double, uint16_t, false>(g, u_row, y_row, kchunk, s, cache.maps, err);
  }
  if (g->id_bytes == 1)
    return g->homog_h ? launch_tma_t<float, uint8_t, true>(g, u_row, y_row, kchunk, s, cache.maps, err)
                      : launch_tma_t<float, uint8_t, false>(g, u_row, y_row, kchunk, s, cache.maps, err);
  return g->homog_h ? launch_tma_t<float, uint16_t, true>(g, u_row, y_row, kchunk, s, cache.maps, err)
                    : launch_tma_t<float, uint16_t, false>(g, u_row, y_row, kchunk, s, cache.maps, err);
}

}  // namespace fdtdmor
