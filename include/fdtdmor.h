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
 * the per-cell material ids (uint8 when nmat <= 255, else uint16), derives the
 * per-axis spacing tables and the per-material update coefficients on the
 * device, and zeroes the fields.  m sources, p probes. */
FDTD_API fdtd_status fdtd_grid_create(const fdtd_grid_desc *desc, int m, const fdtd_port *ports,
                             int p, const fdtd_port *probes, fdtd_stream_t stream,
                             fdtd_grid **out);
FDTD_API fdtd_status fdtd_grid_destroy(fdtd_grid *grid);

/* Replace the material table (same nmat; the per-cell ids are kept), e.g. for
 * an optimisation loop over eps_r.  Host arrays of nmat values; synchronises
 * the stream.  The update coefficients and edge properties follow the new
 * table at the next use. */
FDTD_API fdtd_status fdtd_grid_set_materials(fdtd_grid *grid, int nmat, const double *eps_r, const double *mu_r,
                                    const double *sig_e, const double *sig_m, const uint8_t *pec,
                                    fdtd_stream_t stream);

/* Eq. (CFL): 1/(c sqrt(1/dx^2 + 1/dy^2 + 1/dz^2)) with c = c0/sqrt(min
 * eps_r mu_r) over the non-PEC materials in use and the smallest cell on each
 * axis.  Returns a negative value for a NULL grid. */
FDTD_API double fdtd_cfl_dt(const fdtd_grid *grid);

/* Kernel form of the leap-frog (A2).  All forms compute the same update.
 * AUTO: MARCH on FP32 grids of at least 2^22 cells whose nx is a multiple
 * of 4 and at least 256, SPLIT otherwise.  PERSIST: one launch runs up to
 * 8192 steps in place; its CTAs take (step, half step, z slab, tile) work
 * units in order from a counter and wait (bounded) only for the slabs a unit
 * depends on, so the E and H halves of a slab meet in L2.  SPLIT: an E launch
 * and an H launch per step, each thread updating 4 (FP32) or 2 (FP64)
 * consecutive x cells with vector loads when nx allows.  TMA and FUSED are
 * earlier fused designs kept as reference forms for the parity tests (AUTO
 * never picks them; MARCH supersedes both, about 4x faster than TMA on a
 * 384x384x64 grid): TMA stages planes through shared memory with the tensor
 * memory accelerator, one cell per thread (nx a multiple of 16 for uint8
 * ids, 8 for uint16); FUSED does the same with plain loads.
 * MARCH: one fused pass over memory per step: a CTA marches z over a tile of
 * 7 rows, each thread updating VW consecutive x cells (4 in FP32 on wide
 * grids) with H one plane behind E; the rows exchange E through shared memory
 * (one barrier per plane) and the tile's first row above and +x column are
 * recomputed; in FP32 with 4 cells per thread the plane inputs are staged in
 * shared memory by TMA three planes ahead (rows of the fields and of the
 * material map 16-byte aligned: nx a multiple of 4, and of 16 with uint8
 * material ids); sources and probes follow in one small launch (the step is
 * linear; the sources' terms are gathered once per dt into one term per
 * field value and port).  A staged wait that gives up sets the flag
 * fdtd_check reports. */
typedef enum {
  FDTD_KERNEL_AUTO = 0,
  FDTD_KERNEL_PERSIST = 1,
  FDTD_KERNEL_SPLIT = 2,
  FDTD_KERNEL_TMA = 3,
  FDTD_KERNEL_FUSED = 4,
  FDTD_KERNEL_MARCH = 5
} fdtd_kernel;

/* Choose the kernel form for later fdtd_step calls on this grid.
 * FDTD_EINVAL for an unknown value or TMA on a grid it cannot serve. */
FDTD_API fdtd_status fdtd_grid_set_kernel(fdtd_grid *grid, int kernel);

/* Autotuner of the split form's tile: times trial_steps steps of dt (zero
 * sources) for every x width (1, 2, 4 cells per thread in FP32; 1, 2 in FP64;
 * dividing nx) and every z depth (1, 2, 4, 8 planes per thread), keeps the
 * fastest for later fdtd_step calls on this grid and returns it.  The fields
 * are restored; the call synchronises the stream. */
FDTD_API fdtd_status fdtd_grid_autotune(fdtd_grid *grid, double dt, int trial_steps, int *vw_out, int *lz_out,
                               fdtd_stream_t stream);

/* A2 -- full-order leap-frog, Eq. (matrix) / (MNAform), nsteps steps of dt:
 * E^{n+1} = Ca E^n + Cb (curl H^{n+1/2} - w u^{n+1}),
 * H^{n+3/2} = Da H^{n+1/2} - Db curl E^{n+1}, in the form fdtd_grid_set_kernel
 * chose.
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

/* A11 -- nsteps leap-frog steps of ngrids grids (each with its own dt[q],
 * sources u[q] (device [nsteps][m_q]) and probes y[q] (device [nsteps][p_q],
 * zeroed by the call)) advanced together: per step one E and one H launch for
 * each group of grids sharing field type, id width, uniform mu and x cells per
 * thread, over a work list of every grid's (tile, z range) units, replayed from
 * a captured graph in chunks of 16 steps.  Each grid advances exactly as
 * fdtd_step with its split form would.  reset_fields != 0 zeroes every grid's
 * state first.  u[q] / y[q] may be NULL for grids without sources / probes;
 * u / y may be NULL when no grid has any.  A grid may appear once. */
FDTD_API fdtd_status fdtd_step_batched(fdtd_grid *const *grids, int ngrids, const double *dt, int64_t nsteps,
                              const void *const *u, void *const *y, int reset_fields, fdtd_stream_t stream);

/* (e) -- z planes [k0, k0 + nk) of the six field arrays to / from a buffer
 * laid out [6][nk][ny][nx] in the grid's type (host or device pointer), for
 * the halo exchange of a z-slab decomposition of the grid across GPUs.
 * Asynchronous on the stream; FDTD_EINVAL for planes outside the grid. */
FDTD_API fdtd_status fdtd_planes_get(const fdtd_grid *grid, int k0, int nk, void *dst, fdtd_stream_t stream);
FDTD_API fdtd_status fdtd_planes_set(fdtd_grid *grid, int k0, int nk, const void *src, fdtd_stream_t stream);

/* Field watchdog of fdtd_step / fdtd_step_host (on by default, NaN/Inf
 * only): after each call the squares of the six field arrays are summed in
 * FP64; a sum that is not finite -- a leap-frog run beyond its stability
 * limit, Eq. (singular_limit), overflows -- sets the grid's flag, which
 * fdtd_check reports as FDTD_EUNSTABLE.  growth > 0 also flags a source-free
 * call (no sources, or u = NULL, fields not reset) whose sum grew by more than
 * that factor (the discrete energy x^T R x of Eq. (R_and_F) cannot grow
 * without sources).  sync != 0: fdtd_step synchronises its stream and returns
 * FDTD_EUNSTABLE itself.  enable = 0 switches the watchdog off (one reduction
 * over the fields per call saved). */
FDTD_API fdtd_status fdtd_grid_set_watchdog(fdtd_grid *grid, int enable, double growth, int sync);

/* Polls of a completion-counter wait of the dataflow stepping form
 * (FDTD_KERNEL_PERSIST) before it gives up, sets the grid's flag and returns
 * (fdtd_check then reports FDTD_ETIMEOUT; the fields are not valid).  polls < 0
 * restores the default, 2^24 (about a second).  TMA pipeline waits keep their
 * own fixed limits. */
FDTD_API fdtd_status fdtd_grid_set_wait_limit(fdtd_grid *grid, long long polls);

/* Synchronise the stream and report the grid's flag (then cleared):
 * FDTD_ETIMEOUT if a bounded device-side wait of an earlier fdtd_step gave up
 * (an mbarrier wait of a TMA-staged form, or a completion-counter wait of the
 * dataflow form; the fields are then undefined), FDTD_EUNSTABLE if the field
 * watchdog fired (fdtd_grid_set_watchdog), and, in the checked build
 * (libfdtdmor_checked.so, compiled with -DFDTD_CHECKED), FDTD_ECUDA if a
 * port-list index check of a stepping kernel failed (the access was skipped). */
FDTD_API fdtd_status fdtd_check(fdtd_grid *grid, fdtd_stream_t stream);

/* Copy the six field arrays (Ex, Ey, Ez, Hx, Hy, Hz, each nx*ny*nz of the
 * handle's type, contiguous) to / from the device buffer fields6. */
FDTD_API fdtd_status fdtd_fields_get(const fdtd_grid *grid, void *fields6, fdtd_stream_t stream);
FDTD_API fdtd_status fdtd_fields_set(fdtd_grid *grid, const void *fields6, fdtd_stream_t stream);

/* Per-edge material values the reduction kernels use (A1): 12 arrays of nc
 * values of the grid's type, contiguous -- eps (F/m, 0 on dead edges: walls
 * and PEC) and sigma_e (S/m) for Ex, Ey, Ez, then mu (H/m, 0 for H normal to
 * a wall) and sigma_m for Hx, Hy, Hz -- copied to the device buffer dst. */
FDTD_API fdtd_status fdtd_edge_props_get(fdtd_grid *grid, void *dst, fdtd_stream_t stream);

/* A12 -- gradient of a probe loss L(y) with respect to eps_r by the discrete
 * adjoint of the leap-frog (Eq. (matrix) differentiated exactly; not in the
 * paper).  Runs nsteps steps of dt from zero fields with the sources u
 * (device [nsteps][m], as fdtd_step) keeping ncheckpoints full states
 * (0: ceil(sqrt(nsteps))), then the adjoint recursion -- the same leap-frog
 * with the probes as sources driven by dloss_dy (device [nsteps][p], row n =
 * dL/dy^n) -- back through recomputed segments.  Outputs (device, FP64, either
 * may be NULL): grad_eps_cell[nc] = dL/d eps_r of each cell (the edge
 * permittivity being the area-weighted mean of its four cells, Sec. II-A);
 * grad_eps_mat[nmat] = dL/d eps_r of each material (sum over its cells).
 * Leaves the grid's fields zeroed.  Extra device memory:
 * (K + 4) full states + (c + 1) E fields + 3 nc doubles, c = ceil(nsteps / K). */
FDTD_API fdtd_status fdtd_adjoint(fdtd_grid *grid, double dt, int64_t nsteps, const void *u, const void *dloss_dy,
                         int ncheckpoints, double *grad_eps_cell, double *grad_eps_mat, fdtd_stream_t stream);

/* NEXT-2 -- frequency-domain post-processing (the spectra the paper reads
 * resonances from, Sec. V-A, and S-parameters from, Sec. V-D).
 * fdtd_dft: Y_q(f) = sum_n w_n y^n_q exp(-j 2 pi f t_n) dt, t_n = (n + 1) dt
 * (row n of y samples E^{n+1}), w_n = sin^2(pi (n + 1/2) / nsteps) when
 * hann != 0, else 1.  y: device [nsteps][p] of type prec; freqs: host [nf]
 * (Hz); out: host [p][nf][2] (re, im), FP64.  Synchronises the stream. */
FDTD_API fdtd_status fdtd_dft(const void *y, int64_t nsteps, int p, fdtd_prec prec, double dt, int nf,
                     const double *freqs, int hann, double *out, fdtd_stream_t stream);

/* Resonances: the up to npk largest local maxima of sum_q |Y_q(f)| on nf
 * uniform frequencies in [fmin, fmax] (maxima below rel_floor x the largest
 * are dropped), each refined to the vertex of the parabola through its three
 * samples; returned in ascending order in peaks_hz (host), count in *nfound. */
FDTD_API fdtd_status fdtd_resonances(const void *y, int64_t nsteps, int p, fdtd_prec prec, double dt, double fmin,
                            double fmax, int nf, int hann, double rel_floor, int npk, double *peaks_hz,
                            int *nfound, fdtd_stream_t stream);

/* S-parameters from port waveforms (Sec. V-D): with Y the spectra of y (the
 * structure driven at probe port_in) and Yi those of y_inc (a reference run
 * carrying only the incident wave, e.g. the structure replaced by a matched
 * line), S_q(f) = (Y_q - [q = port_in] Yi_q) / Yi_port_in: S11 at the driven
 * port (reflected over incident), transmission elsewhere.  y, y_inc: device
 * [nsteps][p] of type prec; freqs: host [nf]; out: host [p][nf][2] (re, im),
 * FP64.  FDTD_EINVAL when the incident spectrum is exactly zero at a
 * requested frequency.  Synchronises the stream. */
FDTD_API fdtd_status fdtd_sparams(const void *y, const void *y_inc, int64_t nsteps, int p, fdtd_prec prec, double dt,
                         int nf, const double *freqs, int hann, int port_in, double *out,
                         fdtd_stream_t stream);

/* Kernel launches issued by the calling thread since the last reset (for
 * launch accounting).  fdtd_launch_count(1) returns the count and resets it. */
FDTD_API int64_t fdtd_launch_count(int reset);


/* ------------------------------------------------------------------------
 * Structure-preserving reduction (SPRIM, Sec. II-C) and reduced stepping.
 * ------------------------------------------------------------------------ */
typedef struct mor_basis mor_basis;
typedef struct mor_model mor_model;

/* A3 -- the shifted Schur-complement operator of the Krylov solves (Sec. IV-B,
 * Eqs. (reduced_linear_system_solution1/2)) applied to nb (<= 16) E-field
 * blocks: y_b = S(z_b) x_b with S(z) x = a11 x + z curlH(curlE(x) / a22),
 * a11 = (z-1) eps/dt0 + (z+1) sig/2 and a22 = (z-1) mu/dt0 + (z+1) sig_m/2 per
 * edge -- the rows of A11 - A12 A22^-1 A21 of A(z) = z(R+F) - (R-F) divided
 * by the edge volumes.  z: host [nb][2] (re, im); x, y: device [nb][3][nc]
 * complex values of the grid's type (re, im interleaved), Ex, Ey, Ez; dead
 * edges (walls, PEC) of y are zero.  Allocates one temporary block. */
FDTD_API fdtd_status mor_schur_apply(fdtd_grid *grid, double dt0, int nb, const double *z, const void *x, void *y,
                            fdtd_stream_t stream);

/* Arithmetic of the block Gram-Schmidt (CGS2) products of the basis build:
 * the grid's own type, or tensor-core TF32 / BF16 inputs with FP32
 * accumulation (FDTD_F32 grids only).  Gram norms and R factors are FP64. */
typedef enum { MOR_ORTH_NATIVE = 0, MOR_ORTH_TF32 = 1, MOR_ORTH_BF16 = 2 } mor_orth;

/* A6 / A10 -- Gram product G = A^T diag(w) B of tall column-major FP32
 * matrices, the contraction behind the projection (Eq. (R_and_Freduced)) and
 * the Gram-Schmidt coefficients: A n x M (column stride lda >= n), B n x N
 * (ldb >= n), w n weights or NULL, G M x N row-major FP64 (all device).
 * arith: MOR_ORTH_NATIVE = FP32 CUDA-core products with FP64 sums every 256
 * rows (needs lda = ldb = n); MOR_ORTH_TF32 / MOR_ORTH_BF16 = tcgen05 tensor
 * cores with TF32 / BF16 inputs and FP32 accumulation over row chunks, the
 * chunk sums added in FP64; MOR_GRAM_TF32X3 / MOR_GRAM_BF16X3 = the same in
 * three passes over a head/remainder split of each operand
 * (Ah^T Bh + Ah^T Bl + Al^T Bh), relative error O(2^-20) / O(2^-16) of
 * |A||B| -- the products mor_project uses on the tensor cores.  M, N <= 65535.
 * Synchronises the stream; FDTD_ETIMEOUT if a bounded pipeline wait gave up. */
enum { MOR_GRAM_TF32X3 = 3, MOR_GRAM_BF16X3 = 4 };
FDTD_API fdtd_status mor_gram(int arith, int64_t n, const float *A, int64_t lda, int M, const float *B, int64_t ldb,
                     int N, const float *w, double *G, fdtd_stream_t stream);

/* Krylov solver of the shifted Schur-complement systems.  The paper uses
 * conjugate gradient squared (Sec. IV-B); AUTO picks it for FDTD_F64 grids.
 * CGS and BiCGSTAB are right-preconditioned by the Jacobi diagonal, and
 * convergence is confirmed on the true residual b - S x, with restarts when
 * the recursively updated residual has drifted from it.
 * MOR_SOLVER_COCG (AUTO for FDTD_F32 grids): the Schur complement is complex
 * symmetric, so the conjugate-orthogonal CG applies -- one operator apply per
 * iteration -- with the unconjugated volume-weighted product and the Jacobi
 * diagonal plus one damped Jacobi step on the nodal operator
 * G^T diag(V a11) G for the gradient fields the curl-curl part annihilates.
 * It runs inside an FP64 refinement loop: the true residual bhat - S x is
 * formed in FP64 from an FP64 solution, and the inner COCG (field type) runs
 * to 1e-2 of it until the FP64 residual is below tol.  FP32 arithmetic alone
 * cannot reach tol = 1e-4 on finely graded grids: S magnifies the rounding of
 * x by the ratio of its curl-curl and diagonal parts. */
typedef enum { MOR_SOLVER_AUTO = 0, MOR_SOLVER_CGS = 1, MOR_SOLVER_BICGSTAB = 2, MOR_SOLVER_COCG = 3 } mor_solver;

typedef struct {
  int q;              /* requested columns of V1 and of V2 (Sec. II-C "N~")        */
  int L;              /* expansion points l = -L..L of Eq. (distrib)                */
  double M;           /* radius of the arc, 1.1 in Sec. IV-A                         */
  double fmax;        /* highest frequency of interest (Hz)                          */
  double dt0;         /* time step the basis is built at (> 0)                       */
  int include_center; /* 1: l = -L..L; 0: only the pair z = M e^{+-j 2 pi fmax dt0}   */
  double tol;         /* conjugate-gradient-squared residual limit (Sec. IV-B: 1e-4)  */
  int maxit;          /* iteration cap per shifted solve                             */
  double defl_tol;    /* drop a vector whose norm after CGS2 is below defl_tol x before */
  mor_orth orth;
  mor_solver solver;
} mor_opts;

/* A4 -- the shifted Schur-complement solves of Sec. IV-B on their own: for
 * each of nb (<= 16) points z_b (host [nb][2], re/im) solve
 * S(z_b) x_b = b_b, S the operator of mor_schur_apply at time step
 * opts->dt0, to a relative residual |b - S x| / |b| <= opts->tol, with
 * opts->solver (AUTO: CGS for FDTD_F64 grids, COCG with FP64 refinement for
 * FDTD_F32 grids) and at most opts->maxit iterations per right-hand side.
 * b, x: device [nb][3][nc] complex of the grid's type (x is overwritten).
 * iters, resid: host [nb] or NULL -- iterations and final relative residual
 * per right-hand side (for COCG the FP64 residual of the FP64 solution,
 * before x is rounded to the grid's type).  Returns FDTD_ENOCONV when a
 * right-hand side missed tol (x still written).  Allocates its work
 * vectors; synchronises the stream. */
FDTD_API fdtd_status mor_shifted_solve(fdtd_grid *grid, const mor_opts *opts, int nb, const double *z,
                                       const void *b, void *x, int *iters, double *resid, fdtd_stream_t stream);

/* Fill *opts with M = 1.1, L = 2, tol = 1e-4, maxit = 20000, defl_tol = 1e-8,
 * orth = MOR_ORTH_TF32 (tensor cores on FDTD_F32 grids: TF32 first CGS2 pass,
 * split-precision projection; FDTD_F64 grids always use FP64 products),
 * solver = AUTO -- q, fmax and dt0 must still be set by the caller. */
FDTD_API fdtd_status mor_opts_default(mor_opts *opts);

/* A3-A5 -- SPRIM basis (Sec. II-C, Sec. IV): for each expansion point
 * z_l = M exp(j 2 pi (l/L) fmax dt0), l = 0..L (conjugate points implied), a
 * block-Arnoldi chain of k = q/((2L+1) m) block moments
 * v_0 = A_l^{-1} B, v_j = A_l^{-1} (R+F) v_{j-1}, A_l = z_l (R+F) - (R-F), each
 * shifted solve an iterative solve on the Schur complement
 * A11 - A12 A22^{-1} A21 (Eqs. (reduced_linear_system_solution1/2)) to a
 * normalised residual <= tol, all points and ports of one moment as the
 * right-hand sides of one solve (opts->solver: conjugate gradient squared
 * with Jacobi preconditioning by default on FDTD_F64 grids, COCG with the
 * gradient-corrected preconditioner and FP64 refinement on FDTD_F32 grids,
 * see mor_solver above); then Re/Im of every
 * chain vector is split into its E and H parts and each pool is
 * orthonormalised with CGS2 and deflation -> V1 (3nc x q1), V2 (3nc x q2).
 * Returns FDTD_ENOCONV if a solve hit maxit (the basis is still returned). */
FDTD_API fdtd_status mor_build_basis(fdtd_grid *grid, const mor_opts *opts, fdtd_stream_t stream,
                                     mor_basis **out);
/* Columns kept, worst iteration count and worst final relative residual. */
FDTD_API fdtd_status mor_basis_info(const mor_basis *basis, int *q1, int *q2, int *max_iters,
                                    double *max_resid);
/* Copy V1 (which = 1) or V2 (which = 2), column-major [q][3 nc] of the grid's
 * type, to the device buffer dst. */
FDTD_API fdtd_status mor_basis_get(const mor_basis *basis, int which, void *dst, fdtd_stream_t stream);
FDTD_API fdtd_status mor_basis_destroy(mor_basis *basis);

/* A11 -- n bases built together (batching of Sec. IV over uneven grids):
 * basis i is mor_build_basis(grids[i], &opts[i]) exactly, grid by grid.  The
 * builds run side by side on streams of the library's own (one per host
 * worker, at most FDTDMOR_BATCH_WORKERS, default 8), largest grid first,
 * after the work already queued on `stream`; `stream` then waits for all of
 * them, and each returned basis belongs to `stream` (mor_basis_destroy
 * synchronises it).  grids: n distinct grid handles (the same handle twice is
 * FDTD_EINVAL); opts, out, status: host arrays of n (status may be NULL).
 * out[i] is NULL where build i failed; status[i] is its status.  Returns
 * FDTD_OK, else the worst status (a hard error before FDTD_ENOCONV) with the
 * failing index in fdtd_last_error().  Blocks the calling thread until every
 * build has finished. */
FDTD_API fdtd_status mor_build_basis_batched(int n, fdtd_grid *const *grids, const mor_opts *opts,
                                             fdtd_stream_t stream, mor_basis **out, fdtd_status *status);

/* A6 -- projection, Eq. (R_and_Freduced): D~eps = V1^T D_eps V1,
 * D~se = V1^T D_se V1, D~mu = V2^T D_mu V2, D~sm = V2^T D_sm V2,
 * K~ = V1^T K V2, B~ = V^T B, C~ = C V, accumulated in FP64.  For a basis
 * built with MOR_ORTH_TF32 / MOR_ORTH_BF16 the five Gram products run on the
 * tensor cores in split precision (MOR_GRAM_TF32X3 / MOR_GRAM_BF16X3); else
 * on the CUDA cores in the grid's type. */
FDTD_API fdtd_status mor_project(fdtd_grid *grid, const mor_basis *basis, fdtd_stream_t stream,
                                 mor_model **out);

/* A7 -- perturbation of Sec. III-A for time step dt: with D~eps = Le Le^T,
 * D~mu = Lm Lm^T (Cholesky; equivalent to the symmetric roots), SVD
 * Le^{-1} K~ Lm^{-T} = U S W^T, sigma' = sigma if sigma < gamma 2/dt else
 * gamma 2/dt, K~' = Le U S' W^T Lm^T; then the step matrices of the reduced
 * leap-frog at dt.  *n_clipped receives the number of clipped values (host
 * pointer, may be NULL).  Synchronises the stream. */
FDTD_API fdtd_status mor_perturb(mor_model *model, double dt, double gamma, int *n_clipped,
                                 fdtd_stream_t stream);

/* A8 -- reduced leap-frog, Eq. (reducedMNAform) in block form, nsteps steps at
 * the dt of the last mor_perturb, in one persistent kernel:
 * e <- Pe e - Qe h + be u^{n+1}, h <- Ph h + Qh e + bh u^{n+1}, y^n = C~ e.
 * It runs on a thread-block cluster (up to 16 CTAs) holding row slices of
 * the step matrices in shared memory and exchanging the state through
 * distributed shared memory; where no cluster fits, on one CTA.
 * u: device [nsteps][m], y: device [nsteps][p] (grid type). */
FDTD_API fdtd_status mor_run(mor_model *model, int64_t nsteps, const void *u, void *y,
                             int reset_state, fdtd_stream_t stream);

/* Reduced matrices to host, row-major doubles.  which: 0 D~eps, 1 D~se,
 * 2 D~mu, 3 D~sm, 4 K~, 5 K~' (after mor_perturb), 6 B~_E, 7 C~_E,
 * 8 singular values sigma before clipping (1 x q).  rows/cols receive the
 * shape; host_out may be NULL to query it.  Synchronises the stream. */
FDTD_API fdtd_status mor_model_get(const mor_model *model, int which, double *host_out, int *rows,
                                   int *cols, fdtd_stream_t stream);
FDTD_API fdtd_status mor_model_destroy(mor_model *model);

/* Save a projected model -- D~eps, D~se, D~mu, D~sm, K~ (unperturbed), B~, C~
 * in FP64 and the grid's precision -- to a file, and load it back as a new
 * handle that needs only mor_perturb before mor_run: one reduction serves
 * every time step and excitation, as in the paper's tables, where one MOR
 * time is paired with runs at several s (Tables III, V, VI).  The file holds
 * a magic tag, a version, the sizes and the matrices in the little-endian
 * byte order of the hosts this library builds for.  save synchronises the
 * stream; load returns FDTD_EINVAL for a file it did not write. */
FDTD_API fdtd_status mor_model_save(const mor_model *model, const char *path, fdtd_stream_t stream);
FDTD_API fdtd_status mor_model_load(const char *path, fdtd_stream_t stream, mor_model **out);

/* A12 (reduced model) -- gradient of a probe loss of the reduced leap-frog
 * (Eq. (R_and_Freduced) as prepared by mor_perturb) with respect to eps_r,
 * with the projection V frozen (D~eps = V1^T D_eps V1 is the only reduced
 * matrix that depends on eps; K~ as prepared is held fixed).  Runs nsteps
 * steps from zero state with u (device [nsteps][m]) and the adjoint driven by
 * dloss_dy (device [nsteps][p]); the model, basis and grid must belong
 * together.  Outputs (any may be NULL): grad_eps_cell (device FP64 [nc]),
 * grad_eps_mat (device FP64 [nmat]), grad_De (host FP64 [q1][q1] = dL/dD~eps).
 * Synchronises the stream. */
FDTD_API fdtd_status mor_gradient(mor_model *model, const mor_basis *basis, fdtd_grid *grid, int64_t nsteps,
                         const void *u, const void *dloss_dy, double *grad_eps_cell, double *grad_eps_mat,
                         double *grad_De, fdtd_stream_t stream);

/* A9 -- relative L2 error ||y_red - y_ref[sub]|| / ||y_ref[sub]|| over the
 * common samples: y_red [n][p], y_ref rows offset + i*stride, i < n (device,
 * type prec).  *err receives the value (host).  Synchronises the stream. */
FDTD_API fdtd_status mor_compare(const void *y_red, const void *y_ref, int64_t n, int64_t stride,
                                 int64_t offset, int p, fdtd_prec prec, double *err,
                                 fdtd_stream_t stream);

/* The comparison of mor_compare without any device allocation, for callers
 * that cannot allocate while it runs: a host application or plugin that owns
 * all device memory itself, or a run under an allocator that must not grow.
 * The paper has no counterpart; this is a deployment variant of the A9 step.
 * Arguments and result are those of mor_compare.  Its reduction scratch is a
 * static device array inside the library (64 KiB, held on every device that
 * loads the library until the process exits), so n * p is limited to
 * 16,777,216 samples; larger inputs return FDTD_EINVAL with a message.  The
 * first call on a device looks up the array's device address with
 * cudaGetSymbolAddress; make that first call before any stream capture.
 * Every call overwrites the scratch before reading it (no clearing needed),
 * and calls that overlap on the GPU share it and race: serialise them.
 * Synchronises the stream. */
FDTD_API fdtd_status mor_compare_noalloc(const void *y_red, const void *y_ref, int64_t n, int64_t stride,
                                         int64_t offset, int p, fdtd_prec prec, double *err,
                                         fdtd_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* FDTDMOR_H */
