// A2: the Yee leap-frog of Eq. (matrix) as an E half step and an H half step.
//
// Two launch forms share the per-cell code (e_unit, h_unit):
//  * split (large, HBM-bound grids): per leap-frog step one E launch over the
//    whole grid, then one H launch, ping-ponging between the two field
//    buffers.  Each thread owns one (i, j) column of a 32 x 8 tile and marches
//    over a few planes in z, keeping the plane below (E) or above (H) in
//    registers.
//  * dataflow (yee_stream_kernel): one launch runs many steps in place; CTAs
//    take (step, half, slab, tile) units in order and wait only for the slabs
//    a unit depends on.  Yee updates are in-place safe: the E half reads E only
//    at the edge it writes and H only at neighbours (H is not written in that
//    half), and the H half the other way round.
// Edge coefficients come from a per-cell map of "uniform neighbourhoods"
// (emat): where the eight cells around a cell's E edges share one material the
// kernel takes (Ca, Cb) from the material table, otherwise it averages the
// edge material as in Eq. (matrix).  Sources are added by the CTA owning the
// edge after its E update (block barrier, then an atomic on the global value);
// probes are read in the H half from the final E^{n+1}.
#include <algorithm>
#include <cstdlib>
#include <string>

#include "yee_units.cuh"

namespace fdtdmor {

template <typename T, typename ID, int VW, bool PRE>
__global__ void __launch_bounds__(LTX *LTY, VW >= 4 ? 3 : 4) yee_e_kernel(YeeArgs<T, ID> a, const ID *__restrict__ emat, int lz,
                                                                        int kbase, int kend) {
  wait_prior_grid();
  const int k0 = kbase + blockIdx.z * lz;
  e_unit<T, ID, false, VW, PRE>(a, emat, blockIdx.x, blockIdx.y, k0, min(kend, k0 + lz));
  allow_next_grid();
}

template <typename T, typename ID, bool HOMOG_H, int VW>
__global__ void __launch_bounds__(LTX *LTY) yee_h_kernel(YeeArgs<T, ID> a, int lz, int kbase, int kend) {
  wait_prior_grid();
  const int k0 = kbase + blockIdx.z * lz;
  h_unit<T, ID, HOMOG_H, false, VW>(a, blockIdx.x, blockIdx.y, k0, min(kend, k0 + lz));
  allow_next_grid();
}

// Bounded wait until *c >= target (acquire).  Gives up after `limit` polls
// (2^24 by default, about a second; fdtd_grid_set_wait_limit), or at once when
// another CTA has given up, setting *err; returns false then.
__device__ __forceinline__ bool wait_count(const unsigned *c, unsigned target, unsigned *err, long limit) {
  for (long spins = 0;; ++spins) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
    if (v >= target) return true;
    if ((spins & 31) == 0) {
      unsigned e;
      asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(e) : "l"(err) : "memory");
      if (e) return false;
    }
    if (spins >= limit) {
      atomicOr(err, 2u);
      return false;
    }
    if (spins > 16) __nanosleep(64);
  }
}

// Dataflow form: nsteps leap-frog steps in place on (E, H) = a.Ein = a.Eout,
// a.Hin = a.Hout, without grid-wide barriers.
//
// The grid is cut into nslab z slabs of lz planes; a work unit is one tile of
// one slab in one half step.  Per step the units are ticketed in the order
//   E(0), E(1), H(0), E(2), H(1), ..., E(S-1), H(S-2), H(S-1)
// (each slab's units together), and CTAs take tickets from an atomic counter.
// cnt[1 + s] counts finished E units of slab s and cnt[1 + S + s] finished H
// units, cumulatively over the steps of the launch.  Dependencies, which are
// also the in-place hazards:
//   E(s) of step n needs H(s), H(s-1) of step n-1   (H^{n+1/2} at k and k-1),
//   H(s) of step n needs E(s), E(s+1) of step n     (E^{n+1} at k and k+1).
// Every dependency of a ticket has a smaller ticket, held by a running CTA, so
// the smallest unfinished ticket can always proceed: no co-residency is needed
// and the kernel cannot deadlock.  With the units of neighbouring slabs in
// flight together, E^{n+1} and H^{n+1/2} of a slab are still in L2 when its H
// units run, so DRAM sees each field read once and written once per step.
template <typename T, typename ID, bool HOMOG_H, int VW>
__global__ void __launch_bounds__(LTX *LTY, VW >= 4 ? 2 : 4) yee_stream_kernel(YeeArgs<T, ID> a, const ID *__restrict__ emat, int lz,
                                                              int nslab, int64_t nsteps, const T *u, int m, T *y,
                                                              int p, unsigned *cnt, unsigned *err, long wlimit) {
  __shared__ long long s_ticket;
  __shared__ int s_ok;
  const int tid = threadIdx.y * LTX + threadIdx.x;
  const int ntile = a.ntx * a.nty;
  const long long per_step = 2ll * nslab * ntile;
  const long long total = per_step * nsteps;
  unsigned *ticket = cnt, *doneE = cnt + 1, *doneH = cnt + 1 + nslab;
  for (;;) {
    if (tid == 0) s_ticket = atomicAdd(ticket, 1u);
    __syncthreads();
    const long long t = s_ticket;
    if (t >= total) break;
    const int n = (int)(t / per_step);
    const long long r = t - n * per_step;
    const int b = (int)(r / ntile), tile = (int)(r - (long long)b * ntile);
    // block b of the step: 0 -> E(0); odd b < 2S-1 -> E((b+1)/2); even b -> H(b/2-1); 2S-1 -> H(S-1)
    bool is_e;
    int sl;
    if (b == 0) { is_e = true; sl = 0; }
    else if (b == 2 * nslab - 1) { is_e = false; sl = nslab - 1; }
    else if (b & 1) { is_e = true; sl = (b + 1) / 2; }
    else { is_e = false; sl = b / 2 - 1; }
    if (tid == 0) {
      bool ok = true;
      if (is_e) {
        const unsigned need = (unsigned)n * ntile;
        ok = wait_count(doneH + sl, need, err, wlimit) && (sl == 0 || wait_count(doneH + sl - 1, need, err, wlimit));
      } else {
        const unsigned need = (unsigned)(n + 1) * ntile;
        ok = wait_count(doneE + sl, need, err, wlimit) &&
             (sl + 1 == nslab || wait_count(doneE + sl + 1, need, err, wlimit));
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    const int k0 = sl * lz, k1 = min(a.nz, k0 + lz);
    const int bx = tile % a.ntx, by = tile / a.ntx;
    if (is_e) {
      a.u = u ? u + (int64_t)n * m : nullptr;
      e_unit<T, ID, true, VW>(a, emat, bx, by, k0, k1);
    } else {
      a.y = y ? y + (int64_t)n * p : nullptr;
      h_unit<T, ID, HOMOG_H, true, VW>(a, bx, by, k0, k1);
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(is_e ? doneE + sl : doneH + sl, 1u);
    }
  }
}

// Cells per thread along x: 2 when they divide the rows (every vector load is
// then aligned) and the 32-lane tile is not wider than a row, else 1.
// A tuned width (fdtd_grid_autotune) takes precedence.
int yee_split_vw(const fdtd_grid *g) {
  if (g->tune_vw > 0) return g->tune_vw;
  if (getenv("FDTDMOR_NO_VEC")) return 1;
  // 2 cells per thread: measured faster than 4 (FP32) at the occupancy the
  // register budget allows (fdtd_grid_autotune can pick 4)
  const int v = 2;
  return g->nx % v == 0 && 32 * v <= g->nx ? v : 1;
}

// z planes per thread of the split launches: tuned, else 4 once the grid has
// work for several waves of resident CTAs, else 1.
int yee_split_lz(const fdtd_grid *g) {
  if (g->tune_lz > 0) return std::min(g->nz, g->tune_lz);
  const int vw = yee_split_vw(g);
  const int64_t cols = (int64_t)((g->nx + LTX * vw - 1) / (LTX * vw)) * ((g->ny + LTY - 1) / LTY) * LTX * LTY;
  return std::min(g->nz, env_int("FDTDMOR_LZ", cols * g->nz >= 4ll * 2048 * device_sms() ? 4 : 1));
}


// Per-edge coefficient map for the E launches: on grids whose two field
// buffers and the map (18 values per cell) fit in 64 MB of L2, where the
// material averaging at interfaces, not memory, sets the E launch's time.
bool yee_split_precoef(const fdtd_grid *g) {
  if (const char *e = getenv("FDTDMOR_PRECOEF")) return atoi(e) != 0;
  return (double)g->nc * g->elem * 18.0 <= 64.0 * (1 << 20);
}

// One step as an E launch and an H launch, out of place (fields[cur] ->
// fields[cur ^ 1]).
template <typename T, typename ID, bool HH, int VW>
static fdtd_status launch_split_v(fdtd_grid *g, const void *u_row, void *y_row, cudaStream_t s) {
  FDTD_CHECK(ensure_emat<ID>(g, s));
  YeeArgs<T, ID> a = split_args<T, ID>(g);
  a.u = static_cast<const T *>(u_row);
  a.y = static_cast<T *>(y_row);
  const bool pre = yee_split_precoef(g);
  if (pre) {
    const fdtd_status st = ensure_ecoef<T, ID>(g, a, s);
    FDTD_CHECK(st);
    a.ecoef = g->ecoef.as<T>();
  }
  const int lz = yee_split_lz(g);
  // z slabs ordered E(0), E(1), H(0), E(2), H(1), ...: H of slab s reads the
  // E^{n+1} and H^{n+1/2} of its slab soon after E(s) and E(s + 1) touched
  // them, while they are still in L2 (the kernels are out of place, so any
  // order with H(s) after E(s) and E(s + 1) is exact)
  const int slab = std::max(lz, std::min(g->nz, g->tune_slab > 0 ? g->tune_slab : env_int("FDTDMOR_SLAB", g->nz)));
  const int nslab = (g->nz + slab - 1) / slab;
  const dim3 block(LTX, LTY);
  const ID *emat = g->emat.as<ID>();
  auto E = [&](int q) -> fdtd_status {
    const int kb = q * slab, ke = std::min(g->nz, kb + slab);
    const dim3 grid(g->lists.ntx, g->lists.nty, (ke - kb + lz - 1) / lz);
    if (pre) FDTD_CHECK_CUDA(launch_dependent(yee_e_kernel<T, ID, VW, true>, grid, block, s, a, emat, lz, kb, ke));
    else FDTD_CHECK_CUDA(launch_dependent(yee_e_kernel<T, ID, VW, false>, grid, block, s, a, emat, lz, kb, ke));
    return after_launch("yee_e_kernel");
  };
  auto H = [&](int q) -> fdtd_status {
    const int kb = q * slab, ke = std::min(g->nz, kb + slab);
    const dim3 grid(g->lists.ntx, g->lists.nty, (ke - kb + lz - 1) / lz);
    FDTD_CHECK_CUDA(launch_dependent(yee_h_kernel<T, ID, HH, VW>, grid, block, s, a, lz, kb, ke));
    return after_launch("yee_h_kernel");
  };
  FDTD_CHECK(E(0));
  for (int q = 1; q < nslab; ++q) {
    FDTD_CHECK(E(q));
    FDTD_CHECK(H(q - 1));
  }
  return H(nslab - 1);
}

template <typename T, typename ID, bool HH>
static fdtd_status launch_split_t(fdtd_grid *g, const void *u_row, void *y_row, cudaStream_t s) {
  const int vw = yee_split_vw(g);
  if (sizeof(T) == 4 && vw == 4) return launch_split_v<T, ID, HH, 16 / sizeof(T)>(g, u_row, y_row, s);
  if (vw == 2) return launch_split_v<T, ID, HH, 2>(g, u_row, y_row, s);
  return launch_split_v<T, ID, HH, 1>(g, u_row, y_row, s);
}

// nsteps steps in place on fields[cur], as launches of the dataflow kernel of
// up to kStreamChunk steps each (the counters restart with every launch).
constexpr int64_t kStreamChunk = 8192;

template <typename T, typename ID, bool HH, int VW>
static fdtd_status run_stream_v(fdtd_grid *g, int64_t nsteps, const void *u, void *y, cudaStream_t s) {
  FDTD_CHECK(ensure_emat<ID>(g, s));
  YeeArgs<T, ID> a = split_args<T, ID>(g);
  a.Eout = const_cast<T *>(a.Ein);
  a.Hout = const_cast<T *>(a.Hin);
  auto kern = yee_stream_kernel<T, ID, HH, VW>;
  int occ = 0;
  FDTD_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, LTX * LTY, 0));
  FDTD_REQUIRE(occ >= 1, "yee dataflow kernel: no resident CTA per SM");
  const int cap = occ * device_sms();
  const int ntile = g->lists.ntx * g->lists.nty;
  // one-plane slabs while a step has few units per resident CTA, else four
  int lz = (int64_t)ntile * g->nz <= 4ll * cap ? 1 : 4;
  lz = std::min(g->nz, env_int("FDTDMOR_LZ", lz));
  const int nslab = (g->nz + lz - 1) / lz;
  const int64_t per_step = 2ll * nslab * ntile;
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(kStreamChunk, (int64_t(1) << 31) / per_step));
  FDTD_REQUIRE(per_step < (int64_t(1) << 31), "yee dataflow kernel: grid too large for 32-bit tickets");
  const size_t ncnt = 1 + 2 * (size_t)nslab;
  FDTD_CHECK(g->gsync.alloc(ncnt * sizeof(unsigned), s));
  const int nblk = (int)std::min<int64_t>(cap, per_step * std::min(chunk, nsteps));
  const int m = (int)g->ports.size(), p = (int)g->probes.size();
  const ID *emat = g->emat.as<ID>();
  unsigned *cnt = g->gsync.as<unsigned>(), *err = g->errflag.as<unsigned>();
  for (int64_t n0 = 0; n0 < nsteps; n0 += chunk) {
    const int64_t c = std::min(chunk, nsteps - n0);
    const T *uc = u ? static_cast<const T *>(u) + n0 * m : nullptr;
    T *yc = y ? static_cast<T *>(y) + n0 * p : nullptr;
    FDTD_CHECK_CUDA(cudaMemsetAsync(cnt, 0, ncnt * sizeof(unsigned), s));
    kern<<<nblk, dim3(LTX, LTY), 0, s>>>(a, emat, lz, nslab, c, uc, m, yc, p, cnt, err, (long)g->wait_limit);
    FDTD_CHECK(after_launch("yee_stream_kernel"));
  }
  return FDTD_OK;
}

template <typename T, typename ID, bool HH>
static fdtd_status run_stream_t(fdtd_grid *g, int64_t nsteps, const void *u, void *y, cudaStream_t s) {
  const int vw = yee_split_vw(g);
  if (sizeof(T) == 4 && vw == 4) return run_stream_v<T, ID, HH, 16 / sizeof(T)>(g, nsteps, u, y, s);
  if (vw == 2) return run_stream_v<T, ID, HH, 2>(g, nsteps, u, y, s);
  return run_stream_v<T, ID, HH, 1>(g, nsteps, u, y, s);
}

#define YEE_DISPATCH(FN, ...)                                                                         \
  do {                                                                                               \
    if (g->prec == FDTD_F64) {                                                                       \
      if (g->id_bytes == 1)                                                                          \
        return g->homog_h ? FN<double, uint8_t, true>(__VA_ARGS__) : FN<double, uint8_t, false>(__VA_ARGS__); \
      return g->homog_h ? FN<double, uint16_t, true>(__VA_ARGS__) : FN<double, uint16_t, false>(__VA_ARGS__); \
    }                                                                                                \
    if (g->id_bytes == 1)                                                                            \
      return g->homog_h ? FN<float, uint8_t, true>(__VA_ARGS__) : FN<float, uint8_t, false>(__VA_ARGS__);     \
    return g->homog_h ? FN<float, uint16_t, true>(__VA_ARGS__) : FN<float, uint16_t, false>(__VA_ARGS__);     \
  } while (0)

fdtd_status launch_yee_split(fdtd_grid *g, const void *u_row, void *y_row, cudaStream_t s) {
  YEE_DISPATCH(launch_split_t, g, u_row, y_row, s);
}

fdtd_status run_yee_stream(fdtd_grid *g, int64_t nsteps, const void *u, void *y, cudaStream_t s) {
  YEE_DISPATCH(run_stream_t, g, nsteps, u, y, s);
}

}  // namespace fdtdmor
