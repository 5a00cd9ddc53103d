// Grid helpers used by several translation units.
#pragma once
#include "common.cuh"

namespace fdtdmor {
// Per-material update coefficients (Ca, Cb, Da, Db) for time step dt, cached.
fdtd_status ensure_coef_table(fdtd_grid *g, double dt, cudaStream_t s);
// Per-xy-tile source/probe lists for tiles of tx x ty cells (sources also in
// the +x / +y halo of the neighbouring tile), cached per tile shape.
fdtd_status build_tile_lists(fdtd_grid *g, int tx, int ty, cudaStream_t s);
}  // namespace fdtdmor
