// Grid helpers used by several translation units.
#pragma once
#include "common.cuh"

namespace fdtdmor {
// Per-material update coefficients (Ca, Cb, Da, Db) for time step dt, cached.
fdtd_status ensure_coef_table(fdtd_grid *g, double dt, cudaStream_t s);
// Per-xy-tile source/probe lists for tiles of tx x ty cells (sources also in
// the +x / +y halo of the neighbouring tile), cached per tile shape.
fdtd_status build_tile_lists(fdtd_grid *g, int tx, int ty, cudaStream_t s);
// Field watchdog around a public fdtd_step call (watchdog.cu): energy of the
// fields before a source-free call when a growth limit is set, NaN/Inf and
// growth checks after it (flag bits 4 and 8 of the grid's error flag).
fdtd_status watchdog_before(fdtd_grid *g, const void *u, int reset_fields, cudaStream_t s);
fdtd_status watchdog_after(fdtd_grid *g, const void *u, int reset_fields, cudaStream_t s);
// Edge volume V_e = L_e A~_e of component c at cell (i, j, k) from the axis
// tables (1/primal spacing, 1/dual spacing); 0 for an edge on a wall.
template <typename T>
__device__ __forceinline__ double edge_volume(const T *__restrict__ ax, int nx, int ny, int nz, int c, int i, int j,
                                              int k) {
  const int ntot = nx + ny + nz;
  const int idx[3] = {i, nx + j, nx + ny + k};
  double v = 1.0 / (double)__ldg(ax + AX_RD * ntot + idx[c]);
  for (int a = 0; a < 3; ++a) {
    if (a == c) continue;
    const double r = (double)__ldg(ax + AX_RDD * ntot + idx[a]);
    if (r == 0.0) return 0.0;
    v /= r;
  }
  return v;
}

}  // namespace fdtdmor
