/*
 * fdtdmor.h -- C ABI of the GB300 library for structure-preserving reduction of
 * Yee FDTD equations (Li, Sarris, Triverio, arXiv 1406.7042).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns an fdtd_status; on failure a message is stored in a
 *   thread-local buffer readable with fdtd_last_error().  A failing call leaves
 *   its handles usable.
 * - Handles (fdtd_grid, mor_basis, mor_model) are owned by the library from
 *   *_create / the building call until *_destroy.  Descriptors and host arrays
 *   passed in are copied; the caller may free them when the call returns.
 * - Device pointers (u, y, field buffers) belong to the caller and are used on
 *   the given stream only; calls are asynchronous on that stream unless stated.
 *   A NULL stream means the legacy default stream.
 * - Device memory the library needs for its handles comes from the allocator
 *   installed with fdtd_set_allocator (the Python binding installs PyTorch's
 *   caching allocator), else from cudaMallocAsync/cudaFreeAsync.
 * - Precision: FDTD_F64 handles hold and compute every field in double;
 *   FDTD_F32 handles hold fields in float.  u and y have the handle's type.
 *
 * Storage: six arrays (Ex, Ey, Ez, Hx, Hy, Hz) of nx*ny*nz values each, index
 * (k*ny + j)*nx + i; Ex[k,j,i] at (i+1/2, j, k), Ey at (i, j+1/2, k), Ez at
 * (i, j, k+1/2), Hx at (i, j+1/2, k+1/2), Hy at (i+1/2, j, k+1/2), Hz at
 * (i+1/2, j+1/2, k).  The outer boundary is a PEC box: tangential E on the walls
 * and E on edges touching a PEC cell stay zero.
 */
#ifndef FDTDMOR_H
#define FDTDMOR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FDTD_API __attribute__((visibility("default")))
#else
#define FDTD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *fdtd_stream_t; /* the same type as cudaStream_t */

typedef enum {
  FDTD_OK = 0,
  FDTD_EINVAL = 1,    /* bad argument or descriptor                       */
  FDTD_ENOMEM = 2,    /* device allocation failed                         */
  FDTD_ECUDA = 3,     /* CUDA runtime error                               */
  FDTD_ENOCONV = 4,   /* iterative solver reached its iteration cap       */
  FDTD_EUNSTABLE = 5, /* NaN/Inf or energy-growth watchdog fired          */
  FDTD_ETIMEOUT = 6   /* a bounded device-side wait gave up               */
} fdtd_status;

typedef enum { FDTD_F64 = 0, FDTD_F32 = 1 } fdtd_prec;

/* Grid and materials of Sec. II-A, Eq. (matrix): a rectilinear (possibly
 * non-uniform) grid with per-cell material id.  All pointers are host
 * pointers, copied at create time.  eps_r, mu_r are relative; sig_e (S/m) and
 * sig_m (ohm/m) absolute; pec[m] != 0 marks a perfect electric conductor.
 * Edge permittivity/conductivity is the area-weighted mean of the (up to)
 * four cells sharing the edge; edge permeability the length-weighted mean of
 * the two cells its dual edge crosses. */
typedef struct {
  int nx, ny, nz;
  const double *dx, *dy, *dz; /* cell sizes, lengths nx, ny, nz (metres)  */
  int nmat;                   /* 1..65535                                 */
  const double *eps_r, *mu_r, *sig_e, *sig_m;
  const uint8_t *pec;
  const uint16_t *mat_id;     /* [nz][ny][nx]                             */
  fdtd_prec prec;
} fdtd_grid_desc;

/* One column of B (a source, driven by u, Sec. II-A) or one row of C (a
 * probe): n weighted E edges of one component (0 = Ex, 1 = Ey, 2 = Ez) at
 * linear storage indices cell[] = (k*ny + j)*nx + i.  A source adds
 * -w * u(t) to the electric current balance of its edge (B = -w * edge
 * volume); a probe reads sum w * E.  Edges that are PEC are ignored. */
typedef struct {
  int comp;
  int64_t n;
  const int64_t *cell;
  const double *w;
} fdtd_port;

typedef struct fdtd_grid fdtd_grid;

/* Allocator hooks (optional).  alloc(bytes, stream) returns device memory or
 * NULL; release(ptr, stream) frees it.  Pass NULL, NULL to restore the
 * default (cudaMallocAsync / cudaFreeAsync).  Not thread-safe: call before
 * creating handles. */
typedef void *(*fdtd_alloc_fn)(size_t bytes, fdtd_stream_t stream);
typedef void (*fdtd_free_fn)(void *ptr, fdtd_stream_t stream);
FDTD_API fdtd_status fdtd_set_allocator(fdtd_alloc_fn alloc, fdtd_free_fn release);

FDTD_API const char *fdtd_last_error(void);

/* A1 -- grid and material setup (Sec. II-A): copies the descriptor, uploads
 * the per-cell material ids (uint8 when nmat <= 256, else uint16), derives the
 * per-axis spacing tables and the per-material update coefficients on the
 * device, and zeroes the fields.  m sources, p probes. */
FDTD_API fdtd_status fdtd_grid_create(const fdtd_grid_desc *desc, int m, const fdtd_port *ports,
                             int p, const fdtd_port *probes, fdtd_stream_t stream,
                             fdtd_grid **out);
FDTD_API fdtd_status fdtd_grid_destroy(fdtd_grid *grid);

/* Eq. (CFL): 1/(c sqrt(1/dx^2 + 1/dy^2 + 1/dz^2)) with c = c0/sqrt(min
 * eps_r mu_r) over the non-PEC materials in use and the smallest cell on each
 * axis.  Returns a negative value for a NULL grid. */
FDTD_API double fdtd_cfl_dt(const fdtd_grid *grid);

/* A2 -- full-order leap-frog, Eq. (matrix) / (MNAform), nsteps steps of dt:
 * E^{n+1} = Ca E^n + Cb (curl H^{n+1/2} - w u^{n+1}),
 * H^{n+3/2} = Da H^{n+1/2} - Db curl E^{n+1}, fused in one kernel per step.
 * u: device [nsteps][m], row n = u^{n+1}; y: device [nsteps][p], row n =
 * probes of E^{n+1} (zeroed by the call).  reset_fields != 0 zeroes the state
 * first; otherwise the state continues from the previous call. */
FDTD_API fdtd_status fdtd_step(fdtd_grid *grid, double dt, int64_t nsteps, const void *u, void *y,
                      int reset_fields, fdtd_stream_t stream);

/* The same run with host buffers u_host [nsteps][m] and y_host [nsteps][p]:
 * copies u in, steps, copies y out and synchronises the stream.  u_host and
 * y_host should be pinned for the copies to be asynchronous. */
FDTD_API fdtd_status fdtd_step_host(fdtd_grid *grid, double dt, int64_t nsteps, const void *u_host,
                           void *y_host, int reset_fields, fdtd_stream_t stream);

/* Copy the six field arrays (Ex, Ey, Ez, Hx, Hy, Hz, each nx*ny*nz of the
 * handle's type, contiguous) to / from the device buffer fields6. */
FDTD_API fdtd_status fdtd_fields_get(const fdtd_grid *grid, void *fields6, fdtd_stream_t stream);
FDTD_API fdtd_status fdtd_fields_set(fdtd_grid *grid, const void *fields6, fdtd_stream_t stream);

/* Kernel launches issued by the calling thread since the last reset (for
 * launch accounting).  fdtd_launch_count(1) returns the count and resets it. */
FDTD_API int64_t fdtd_launch_count(int reset);

#ifdef __cplusplus
}
#endif
#endif /* FDTDMOR_H */
