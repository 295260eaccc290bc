/*
 * qmcspl.h -- C ABI of the GB300 (sm_103a) planewave-orbital spline library.
 *
 * The library evaluates single-particle orbitals given as planewave sums
 *     phi_n(r) = sum_G c_{G n} exp(i G.r)                        (paper Eq. pw_orbital)
 * with their Cartesian gradients and Laplacians at many electron positions, through
 * a tricubic polynomial basis on a periodic grid (Parker, Umrigar, Alfe, Hennig,
 * Wilkins, arXiv:1309.6250, Sec. II and the Appendix):
 *   - smoothing B-splines, Eq. (b-splinecoefficients)          QMCSPL_BSPLINE_SMOOTH
 *   - interpolating B-splines, Appendix "Interpolating ..."    QMCSPL_BSPLINE_INTERP
 *   - cubic Lagrange interpolation, Eq. (lagrangeinterpolation3), with the separate
 *     gradient and Laplacian tables of Sec. III C            QMCSPL_LAGRANGE
 *   - cubic pp-splines, Eq. (pp-splineinterpolation3)          QMCSPL_PPSPLINE
 * B-splines may carry the separate Laplacian table recommended in Sec. III A / IV.
 *
 * Conventions shared by every call
 *   - Status: every call returns QMCSPL_OK (0) or one of the QMCSPL_ERR_* codes;
 *     qmcspl_last_error() then gives a message (per calling thread).  Arguments are
 *     validated before anything is launched; on an error nothing is written.
 *   - Pointers named *_host are host memory; all other array pointers of the eval
 *     calls are device memory of the device the handle was created on.  The caller
 *     owns every buffer it passes; the library owns the coefficient tables.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device work is
 *     asynchronous on that stream unless a call says otherwise.  Errors a kernel
 *     detects on the device (a non-finite position) are recorded in the handle and
 *     reported by qmcspl_sync().
 *   - Threads: calls on different handles may run concurrently; calls on one handle must
 *     not (a handle owns scratch memory that its evaluations reuse).
 *   - Lattice: row-major 3x3 with the lattice vectors a_1, a_2, a_3 as COLUMNS (bohr),
 *     so r = a s for crystal coordinates s.  Positions may lie anywhere; they are
 *     wrapped into the cell (Eq. reducedcoordinate).
 *   - Output dtype: double for QMCSPL_F64 and QMCSPL_DF64 tables, float for QMCSPL_F32 /
 *     QMCSPL_BF16.
 *     Output layouts (P positions, O orbitals, row-major):
 *         val [P][O],   grad [P][3][O] (Cartesian x, y, z),   lap [P][O].
 *     For a Bloch handle (opts.bloch = 1) every element is a complex number stored as
 *     (re, im), i.e. the same layouts with a trailing [2]: val [P][O][2],
 *     grad [P][3][O][2], lap [P][O][2] (the layout of complex64 / complex128 arrays).
 */
#ifndef QMCSPL_H
#define QMCSPL_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qmcspl_s* qmcspl_t;   /* opaque handle owning the coefficient tables */

enum qmcspl_status {
    QMCSPL_OK = 0,
    QMCSPL_ERR_ARG = 1,            /* invalid argument (null pointer, size, enum value) */
    QMCSPL_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    QMCSPL_ERR_OOM = 3,            /* device or host allocation failed */
    QMCSPL_ERR_UNSUPPORTED = 4,    /* combination not supported (e.g. batched degree-n handles) */
    QMCSPL_ERR_TIMEOUT = 5,        /* a bounded device wait gave up */
    QMCSPL_ERR_NOT_HERMITIAN = 6,  /* coefficients do not give a real (Gamma-point) orbital */
    QMCSPL_ERR_DEVICE = 7          /* a kernel flagged bad input (non-finite position) */
};

enum qmcspl_method {
    QMCSPL_BSPLINE_SMOOTH = 0,     /* Eq. (b-splinecoefficients): beta = sum c_G/gamma_G e^{iG.x} */
    QMCSPL_BSPLINE_INTERP = 1,     /* interpolating B-spline (cyclic tridiagonal system) */
    QMCSPL_LAGRANGE = 2,           /* cubic Lagrange, five tables (phi, grad phi, lap phi) */
    QMCSPL_PPSPLINE = 3            /* cubic pp-spline, eight coefficients per grid point */
};

enum qmcspl_storage {
    QMCSPL_F64 = 0,                /* tables and arithmetic in double */
    QMCSPL_F32 = 1,                /* float tables, float accumulation */
    QMCSPL_BF16 = 2,               /* bfloat16 tables, float accumulation */
    QMCSPL_DF64 = 3                /* double-float: each coefficient a pair of floats whose
                                      sum carries ~48 significant bits, arithmetic in
                                      error-free FP32 pair operations, double outputs; the
                                      accuracy class of FP64 at FP32-pipe speed.  Cubic
                                      B-splines on uniform grids (with or without separate
                                      Laplacian and gradient tables); their backward pass
                                      runs in FP64 on the stored pairs.  Lagrange, pp and
                                      B-splines of other degrees or on graded grids
                                      reject it (QMCSPL_ERR_UNSUPPORTED). */
};

typedef struct {
    int method;        /* enum qmcspl_method */
    int storage;       /* enum qmcspl_storage */
    int separate_lap;  /* B-splines: 1 = also build the Laplacian table (Sec. III C,
                          memory x2) and return its value as the Laplacian; 0 = the
                          Laplacian of the spline itself.  Ignored by Lagrange (always
                          its own Laplacian table) and pp (always the spline's own). */
    int lanes;         /* threads that share one position in the evaluation kernels,
                          each owning one 16-byte chunk of every stored row: 0 = choose
                          automatically, else 1, 2, 4, 8, 16 or 32.  Rows are padded to
                          a multiple of lanes x 16 bytes. */
    int separate_grad; /* B-splines: 1 = also build tables of d_x phi, d_y phi, d_z phi (the
                          separate gradient approximations of Sec. III C; requires
                          separate_lap = 1, five tables in all, memory x5) and return
                          their values as the gradient.  Ignored by Lagrange (always
                          five tables) and pp. */
    int bloch;         /* 0 = real Gamma-point orbitals (Hermitian coefficients, real
                          outputs).  1 = complex Bloch orbitals at crystal momentum k
                          (Sec. II): phi_n(r) = u_n(r) exp(i k.r) with the periodic part
                          u_n(r) = sum_G c_{G n} exp(i G.r), so the planewave sum is
                          sum_G c_{G n} exp(i (k+G).r).  No symmetry is required of the
                          coefficients; Re u_n and Im u_n are tabulated as two adjacent
                          real functions (twice the table memory of n_orb real orbitals)
                          and every output is complex (see qmcspl_eval_vgl). */
    double kpoint[3];  /* bloch = 1: k in units of the reciprocal lattice vectors,
                          k = 2 pi a^{-T} kpoint (Cartesian, 1/bohr).  Ignored when
                          bloch = 0. */
} qmcspl_opts;

typedef struct {
    int dims[3];             /* grid points along a_1, a_2, a_3 */
    int n_orb;               /* orbitals */
    int n_orb_padded;        /* orbitals per stored row (zero padded) */
    int method, storage, separate_lap;
    int n_tables;            /* value tables stored: 1, 2 (B-spline + Laplacian), 5 (Lagrange, or
                                B-spline with separate gradient tables), or 1 pp table of 8 entries */
    int entries_per_point;   /* stored values per grid point per orbital row: 1, or 8 (pp) */
    int rows_z;              /* stored z planes per (x, y) column (periodic ghost planes included) */
    int lanes;               /* threads sharing one position in the eval kernel */
    int tiles;               /* orbital tiles per position */
    long long table_bytes;   /* device bytes of all coefficient tables */
    long long n_pw;          /* planewaves the tables were built from */
    int bloch;               /* 1: complex Bloch orbitals (n_orb complex orbitals, stored as
                                2 n_orb real functions per row: Re u_0, Im u_0, Re u_1, ...) */
    double kpoint[3];        /* k in units of the reciprocal lattice vectors (bloch = 1) */
    int separate_grad;       /* 1: B-spline with separate gradient tables */
    int degree;              /* B-spline degree (3 unless created by qmcspl_create_grid) */
    int nonuniform;          /* 1: per-axis grid points (qmcspl_create_grid) */
    int staged;              /* 1: pencil order evaluates with the shared-memory-staged kernel
                                (see qmcspl_set_order); 0: it falls back to cell order */
    int block_threads;       /* block shape set by qmcspl_set_block (0 = automatic) */
} qmcspl_info_t;

/*
 * qmcspl_create -- build the coefficient tables of n_orb real orbitals.
 *
 * Paper: Eq. (pw_orbital) defines the input; the Appendix defines the tables:
 * smoothing coefficients by Eq. (b-splinecoefficients), interpolating coefficients by
 * the periodic system of "Interpolating B-spline coefficients", Lagrange tables as the
 * grid values of phi, its gradient and Laplacian, pp tables by
 * Eq. (pp-splinecoefficients3).
 *
 *   out      [out] receives the handle (set to NULL on failure)
 *   lattice  host double[9], row-major, columns = lattice vectors (bohr); non-singular
 *   dims     host int[3], grid points per lattice vector, each in [4, 4096]
 *   n_pw     number of planewaves, >= 1
 *   miller   host int[n_pw][3], integer Miller indices n of G = 2 pi a^{-T} n; each
 *            G must appear once and (real orbitals) -G must be present
 *   n_orb    number of orbitals, >= 1 (complex orbitals for a Bloch handle)
 *   coef     host double[n_orb][n_pw][2], (re, im) of c_{G n}; real orbitals must
 *            satisfy c_{-G} = conj(c_G) to 1e-12 relative, else
 *            QMCSPL_ERR_NOT_HERMITIAN; Bloch orbitals have no such condition
 *   opts     host pointer to the options (method, storage, separate_lap, lanes, bloch,
 *            kpoint).  For a Bloch handle the separate derivative tables approximate
 *            the periodic parts of the derivatives of phi itself: the Laplacian table
 *            (B-splines with separate_lap, Lagrange) is built from -|k+G|^2 c_G and
 *            the Lagrange gradient tables from i (k+G) c_G.
 *   stream   cudaStream_t the construction runs on; the call blocks until the tables
 *            are complete, then frees its temporaries
 *
 * The tables live on the current CUDA device.  The construction arithmetic (frequency
 * grid, symbol division, inverse transforms) is FP64 whatever the storage type.
 */
int qmcspl_create(qmcspl_t* out, const double lattice[9], const int dims[3], int n_pw,
                  const int* miller, int n_orb, const double* coef, const qmcspl_opts* opts,
                  void* stream);

/*
 * qmcspl_create_grid -- qmcspl_create for B-splines of another odd degree, and interpolating
 * B-splines of any of these degrees on a non-uniform grid.
 *
 * Paper: Sec. II, "Common features" (each method may use polynomials of any order n; the
 * paper uses cubics) and "Grid" (uniform or non-uniform grids); Appendix, the B-spline
 * recurrence and "Interpolating B-spline coefficients" (interpolation needs no evenly
 * spaced grid).  The basis of grid point m is the recurrence's b_j^n centred on x_m, with
 * the degree-0 constant C_n = 1 / B_n(0) so that it peaks at one (C_3 = 3/2 as in the paper;
 * C_1 = 1, C_5 = 20/11, C_7 = 315/151).  The coefficients interpolate phi (and, with
 * separate_lap, lap phi) at every grid point.
 *
 *   grid->degree    1, 3, 5 or 7 (0 = 3).  Uniform grids: the periodic system is solved
 *                   exactly in Fourier space (its symbol sum_j C_n B_n(j) e^{i j th}).
 *   grid->knots[a]  NULL for a uniform axis, else host double[dims[a]]: the grid points of
 *                   axis a in reduced coordinates, strictly increasing in [0, 1); either
 *                   all three axes or none.  Any of the four degrees; the planewave band
 *                   must fit the grid (dims[a] >= 2 max|n_a| + 1, else QMCSPL_ERR_ARG).  The
 *                   periodic interpolation system is solved along each axis in FP64: cyclic
 *                   tridiagonal for the cubic, the identity for degree 1, and for degrees 5
 *                   and 7 through the inverse of the cyclic banded matrix (computed on the
 *                   host, O(N^3) per axis; QMCSPL_ERR_ARG if it is singular).
 * Other arguments as qmcspl_create; opts->method QMCSPL_BSPLINE_INTERP, or on uniform
 * grids also QMCSPL_BSPLINE_SMOOTH (Eq. b-splinecoefficients with gamma the Fourier
 * transform of the degree-n basis, C_n sinc^{n+1}(th/2) per axis); storage F64, F32 or BF16;
 * separate_grad 0 (else QMCSPL_ERR_UNSUPPORTED); Bloch orbitals are accepted.
 * dims[a] >= degree + 1.  Evaluation (qmcspl_eval_vgl, _host, _noalloc) and the backward
 * pass have the same outputs and arguments; the stencil is (n + 1)^3 points.  Batched
 * evaluation is not available for these handles (QMCSPL_ERR_UNSUPPORTED).  grid = NULL is
 * qmcspl_create.
 */
typedef struct {
    int degree;
    const double* knots[3];
} qmcspl_grid_opts;
int qmcspl_create_grid(qmcspl_t* out, const double lattice[9], const int dims[3], int n_pw,
                       const int* miller, int n_orb, const double* coef, const qmcspl_opts* opts,
                       const qmcspl_grid_opts* grid, void* stream);

/* qmcspl_destroy -- synchronise the device and free the handle and its tables.
 * NULL is accepted. */
int qmcspl_destroy(qmcspl_t h);

/* qmcspl_info -- describe a handle (host struct filled in). */
int qmcspl_info(qmcspl_t h, qmcspl_info_t* out);

/*
 * qmcspl_eval_vgl -- value, Cartesian gradient and Laplacian of every orbital at
 * every position.
 *
 * Paper: Eq. (reducedcoordinate) maps r to a grid cell and t in [0,1)^3; the tricubic
 * sum of Eq. (b-splineapproximation) / (lagrangeinterpolation3) /
 * (pp-splineinterpolation3) gives the value and reduced derivatives; the chain rule
 * of Sec. II (Coordinates) gives grad = N_i (a^-1)^T grad_t and
 * lap = sum_ij N_i N_j (a^-1 a^-T)_ij d2/dt_i dt_j.  With a separate Laplacian table
 * (B-splines) or for Lagrange, lap is the interpolated table; with separate gradient
 * tables (Lagrange, B-splines with separate_grad) so is grad.
 * Bloch handles (Sec. II): with c + i s = exp(i k.r) at the unwrapped position r,
 *   phi = (c + i s) u,   grad phi = (c + i s)(grad u + i k u),
 *   lap phi = (c + i s)(lap u + 2 i k.grad u - |k|^2 u),
 * where a separate table replaces the bracket by its own interpolated value.  The
 * factor is computed once per position in FP64.
 *
 *   pos    device double[n_pos][3], Cartesian (bohr); non-finite entries give NaN
 *          outputs for that position and QMCSPL_ERR_DEVICE at qmcspl_sync
 *   n_pos  >= 0 (0 is a no-op)
 *   val, grad, lap  device outputs in the layouts above (double for F64 tables, float
 *          otherwise); any of them may be NULL to skip it
 *   stream cudaStream_t; asynchronous
 */
int qmcspl_eval_vgl(qmcspl_t h, const double* pos, long long n_pos, void* val, void* grad,
                    void* lap, void* stream);

/*
 * qmcspl_eval_vgl_host -- qmcspl_eval_vgl from and to HOST memory.
 *
 * Same computation; the library stages the positions to the device and the outputs
 * back in chunks, overlapping copies and kernels on internal streams ordered after
 * `stream`.  Blocking: on return the host outputs are complete.  For full copy speed
 * the host buffers should be page-locked (cudaHostAlloc / pinned torch tensors).
 * Device staging buffers are allocated on first use and kept by the handle.
 */
int qmcspl_eval_vgl_host(qmcspl_t h, const double* pos_host, long long n_pos, void* val_host,
                         void* grad_host, void* lap_host, void* stream);

/*
 * qmcspl_eval_vgl_host_ex -- qmcspl_eval_vgl_host with a choice of output type.
 *
 * Not in the paper.  The host-buffer evaluation moves every output across the host link, which
 * bounds it (about 180 GB/s device-to-host, against the kernels' rate of some TB/s).  With a
 * 16-bit output type each chunk of outputs is converted on the device (round to nearest even)
 * before it is copied, halving the bytes:
 *   opts->out_type  QMCSPL_OUT_NATIVE: the output dtype of qmcspl_eval_vgl (opts = NULL too);
 *                   QMCSPL_OUT_BF16: bfloat16 (8 significant bits: relative rounding 2^-9, the
 *                   float exponent range); QMCSPL_OUT_F16: IEEE half (11 significant bits:
 *                   relative 2^-12, but magnitudes above 65504 become infinities)
 *   val_host, grad_host, lap_host  host buffers in the usual layouts, 2-byte elements for the
 *                   16-bit types; any may be NULL to skip that output (no conversion, no copy)
 * The 16-bit types are for real orbitals with float or bfloat16 tables (else
 * QMCSPL_ERR_UNSUPPORTED).  The device staging buffers for the converted chunks (2 x 5 x 65536 x
 * n_orb x 2 bytes) are allocated on first use and kept by the handle.
 */
enum qmcspl_out_type {
    QMCSPL_OUT_NATIVE = 0,
    QMCSPL_OUT_BF16 = 1,
    QMCSPL_OUT_F16 = 2
};
typedef struct {
    int out_type;    /* enum qmcspl_out_type */
} qmcspl_host_opts;
int qmcspl_eval_vgl_host_ex(qmcspl_t h, const double* pos_host, long long n_pos, void* val_host,
                            void* grad_host, void* lap_host, const qmcspl_host_opts* opts, void* stream);

/*
 * qmcspl_eval_vgl_backward -- adjoint of qmcspl_eval_vgl (every method, degree and grid).
 *
 * Not in the paper: for a scalar loss L with upstream gradients gv = dL/dval,
 * gg = dL/dgrad, gl = dL/dlap (same layouts and dtype as the outputs; any may be NULL
 * meaning zero) it gives
 *   dcoef     device, canonical layout [Nx][Ny][Nz][O] (unpadded, no ghost planes),
 *             output dtype; ACCUMULATED (+=) with dL/dbeta of the value table.
 *             NULL skips the coefficient adjoint.
 *   dcoef_lap same for the separate Laplacian table (required iff separate_lap and
 *             dcoef is given; must be NULL otherwise).
 *   dpos      device double[n_pos][3], WRITTEN with dL/dr.  NULL skips it.
 * The coefficient adjoint scatters into 64 stencil rows per position with atomic
 * adds, so its summation order (and last bits) vary from run to run.
 * Bloch handles (complex outputs z): gv, gg, gl hold g = dL/dRe z + i dL/dIm z in the
 * complex output layouts ([P][O][2], [P][3][O][2], [P][O][2]); dcoef and dcoef_lap are the
 * gradients of the stored tables of Re u and Im u, canonical layout [Nx][Ny][Nz][O][2]; dpos
 * includes the derivative of the phase exp(i k.r).
 * Five-table handles (Lagrange, and B-splines with separate_grad): the outputs are the values
 * of the tables phi, d_x phi, d_y phi, d_z phi, lap phi with one set of weights, so dcoef is
 * [5][Nx][Ny][Nz][O] (those tables in that order, canonical layout) and dcoef_lap must be NULL.
 * pp handles: dcoef is [8][Nx][Ny][Nz][O], sigma^{kappa mu nu} at index 4(kappa-1) + 2(mu-1) +
 * (nu-1) as in qmcspl_get_table; dcoef_lap must be NULL.
 * Double-float tables: the adjoint runs in FP64 on the stored pairs (hi + lo) read as
 * doubles; dcoef is double (the output dtype).  B-splines of degree 1, 5, 7 and on graded
 * grids: the same adjoints over their (n + 1)^3-point stencils (a scalar kernel).
 */
int qmcspl_eval_vgl_backward(qmcspl_t h, const double* pos, long long n_pos, const void* gv,
                             const void* gg, const void* gl, void* dcoef, void* dcoef_lap,
                             double* dpos, void* stream);

/*
 * qmcspl_eval_batched -- qmcspl_eval_vgl for several handles in one call.
 *
 * Walkers of cells with different orbital counts and grids go through one batched
 * launch whose work list spreads every cell's positions evenly over the whole GPU (each
 * warp task moves the same number of bytes whatever the cell).  A cell with enough work
 * to fill the GPU for at least four rounds of warp tasks on its own instead gets its own
 * launch, with the launch shape qmcspl_eval_vgl would use (large launches lose little to
 * their last, partly filled round, and the single-cell shape is faster); all launches of
 * a call go to `stream` in cell order.  All handles must be
 * B-spline handles without separate gradient tables on one device with the same
 * storage type, the same separate_lap setting and the same bloch setting (k points may
 * differ per cell).
 *   n_cells   1..QMCSPL_MAX_BATCH
 *   h         host array of n_cells distinct handles (a cell's visiting order is kept in its
 *             handle's scratch, so a handle given twice is refused with QMCSPL_ERR_ARG)
 *   pos, val, grad, lap   host arrays of n_cells DEVICE pointers (layouts as above;
 *             val/grad/lap entries may be NULL)
 *   n_pos     host array of n_cells position counts
 * Asynchronous on `stream`.  The cell descriptors travel as kernel parameters (no
 * copy).  Each handle's evaluation order applies (qmcspl_set_order): cells evaluated
 * in cell order are sorted first by three small kernels per cell, in the handle's
 * scratch memory, which a call allocates only when a cell has more positions than
 * any earlier call on that handle.  After one call at the largest sizes the call
 * allocates nothing and can be captured in a CUDA graph.
 */
#define QMCSPL_MAX_BATCH 48
int qmcspl_eval_batched(int n_cells, const qmcspl_t* h, const double* const* pos,
                        const long long* n_pos, void* const* val, void* const* grad,
                        void* const* lap, void* stream);

/*
 * qmcspl_eval_batched_ex -- qmcspl_eval_batched with an explicit launch plan.
 *
 * Not in the paper (the cost model it serves is Sec. III B's: every evaluation gathers 64
 * coefficient rows, whatever the cell).  opts = NULL is qmcspl_eval_batched.
 *   opts->launch   QMCSPL_BATCH_AUTO: the rule of qmcspl_eval_batched;
 *                  QMCSPL_BATCH_SINGLE: every cell's evaluation in the one persistent batched
 *                  launch (the cells' warp tasks back to back in one static work list);
 *                  QMCSPL_BATCH_SPLIT: one launch per cell, each with its handle's block shape
 *   opts->threads  block shape of the batched launch: 0 (= 512) or 512, or 640 for float and
 *                  bfloat16 tables (else QMCSPL_ERR_UNSUPPORTED)
 * The cell-order sorting runs per cell before the evaluation launches, as in
 * qmcspl_eval_batched; the results do not depend on the plan (each position is computed the
 * same way).  Other arguments and conditions as qmcspl_eval_batched.
 */
enum qmcspl_batch_launch {
    QMCSPL_BATCH_AUTO = 0,
    QMCSPL_BATCH_SINGLE = 1,
    QMCSPL_BATCH_SPLIT = 2
};
typedef struct {
    int launch;      /* enum qmcspl_batch_launch */
    int threads;     /* 0, 512 or 640 */
} qmcspl_batch_opts;
int qmcspl_eval_batched_ex(int n_cells, const qmcspl_t* h, const double* const* pos,
                           const long long* n_pos, void* const* val, void* const* grad,
                           void* const* lap, const qmcspl_batch_opts* opts, void* stream);

/*
 * qmcspl_set_block -- block shape of the tricubic B-spline evaluation kernel for this handle.
 *
 * Not in the paper.  The kernel walks a static list of warp tasks (one position and one
 * orbital tile per group of lanes) with one thread block per SM, so the block shape sets how
 * many neighbouring positions share an SM's L1 at a time (threads / lanes positions per block)
 * and how many registers each thread may use.  0 = automatic: 640 threads for float tables with
 * the Laplacian table on launches of four or more rounds of warp tasks, 512 otherwise; 512 or
 * 640 (float and bfloat16 tables only) fixes the shape.  Results do not depend on it.  The
 * autotuner (paper_1309_6250_gb300/autotune.py) picks it per workload.
 */
int qmcspl_set_block(qmcspl_t h, int threads);

/*
 * qmcspl_get_table -- copy one stored table back to the host in canonical layout
 * double[Nx][Ny][Nz][O] (padding and ghost planes removed, converted to double); a
 * Bloch handle gives double[Nx][Ny][Nz][O][2], (Re, Im) of the tabulated periodic part.
 *   table  B-splines: 0 = coefficients, 1 = Laplacian coefficients (separate_lap);
 *          Lagrange, and B-splines with separate_grad: 0..4 = tables of phi, d_x phi,
 *          d_y phi, d_z phi, lap phi;
 *          pp: 0..7 = sigma^{kappa mu nu} with index 4(kappa-1) + 2(mu-1) + (nu-1).
 * Blocking.
 */
int qmcspl_get_table(qmcspl_t h, int table, double* out_host, void* stream);

/*
 * qmcspl_set_table -- overwrite one stored table from a DEVICE array in canonical layout.
 *
 * Not in the paper: it makes the coefficient gradient of qmcspl_eval_vgl_backward usable for
 * optimising the orbitals, since the coefficients of Eq. (b-splineapproximation) (and of the
 * other bases) can then be changed between evaluations without rebuilding the handle.  The
 * inverse of qmcspl_get_table:
 *   table      the same numbering as qmcspl_get_table (B-splines 0 = coefficients, 1 = Laplacian
 *              coefficients; five-table handles 0..4; pp 0..7 = the sigma entries)
 *   src        device array [Nx][Ny][Nz][O] (a Bloch handle: [Nx][Ny][Nz][O][2], Re and Im of the
 *              tabulated periodic part), unpadded, without ghost planes, of src_dtype
 *   src_dtype  QMCSPL_F64 (double) or QMCSPL_F32 (float)
 *   stream     cudaStream_t; asynchronous: src must stay valid and unchanged until the work on
 *              `stream` is done, and evaluations of the handle on other streams must be ordered
 *              after it by the caller
 * Each value is converted to the storage type exactly as the construction converts its FP64
 * coefficients (round to nearest; double-float: hi = rounded value, lo = rounded remainder),
 * the periodic ghost planes are rewritten and the row padding stays zero, so that
 * qmcspl_set_table(h, t, table from qmcspl_get_table) leaves the handle bit for bit as it was.
 * The handle's planewave description is not updated: the tables are what evaluation uses.
 */
int qmcspl_set_table(qmcspl_t h, int table, const void* src, int src_dtype, void* stream);

/*
 * qmcspl_set_order -- choose the order in which qmcspl_eval_vgl visits positions.
 *
 * Not in the paper.  Results do not depend on it (each position is computed the same
 * way; outputs are always written in input order).  Visiting positions grouped by
 * grid cell lets neighbouring positions share their stencil rows in the on-chip
 * caches instead of re-reading them from HBM.  Cell order sorts the positions into
 * spatial bins first (a counting sort on the device, in scratch memory the handle
 * allocates on first use and grows when a call has more positions).
 * Pencil order sorts them into columns of 2 x 2 grid cells in (x, y), each by z cell, and
 * evaluates them with the staged kernel: each z plane of the 5 x 5 stencil columns of a
 * pencil is copied into shared memory once (tiled tensor copies) and read there by every
 * position of the pencil that needs it.  It applies to cubic B-splines on uniform grids
 * with FP32 or BF16 tables, without separate gradient tables, whose rows are 128, 256 or
 * 512 bytes with one 16-byte chunk per lane (32, 64 or 128 FP32 orbitals; 64, 128 or 256
 * BF16 orbitals); other handles, the batched call and qmcspl_eval_vgl_noalloc take cell
 * order instead.  On GB300 cell order is the faster of the two for every workload measured,
 * so pencil order is never chosen automatically.
 *   mode  QMCSPL_ORDER_AUTO (default: cell order from 8192 positions on when the tables are
 *         larger than the L2 cache; for tables that fit in L2, once the positions per bin of
 *         4 x 4 x 4 cells reach 8, 32 or 192 for tables filling more than 60 %, more than 30 %
 *         or at most 30 % of L2 -- below that the table is gathered from L2 in input order
 *         about as fast, without the sort), QMCSPL_ORDER_INPUT, QMCSPL_ORDER_CELL or
 *         QMCSPL_ORDER_PENCIL
 * A staged evaluation whose pipeline stalls for about a second (a fault of this library,
 * not of the input) gives up; qmcspl_sync then returns QMCSPL_ERR_TIMEOUT.
 */
enum qmcspl_order {
    QMCSPL_ORDER_AUTO = 0,
    QMCSPL_ORDER_INPUT = 1,
    QMCSPL_ORDER_CELL = 2,
    QMCSPL_ORDER_PENCIL = 3
};
int qmcspl_set_order(qmcspl_t h, int mode);

/*
 * qmcspl_get_order -- the order in which qmcspl_eval_vgl (and the backward pass) would visit
 * n_pos positions: QMCSPL_ORDER_INPUT, QMCSPL_ORDER_CELL or QMCSPL_ORDER_PENCIL, with
 * QMCSPL_ORDER_AUTO resolved.  Not in the paper.
 *   order  host int receiving the order
 * QMCSPL_ERR_ARG for a NULL handle or order or n_pos < 0.  No device work.
 */
int qmcspl_get_order(qmcspl_t h, long long n_pos, int* order);

/*
 * qmcspl_eval_vgl_noalloc -- qmcspl_eval_vgl in cell order, allocating nothing.
 *
 * The paper has no counterpart; this is a service for callers that cannot allocate
 * device memory while they evaluate: programs that give all device memory to their own
 * pool allocator at start-up, and time-critical loops that must not call cudaMalloc or
 * cudaFree (which can block the whole device).  It computes exactly what
 * qmcspl_eval_vgl computes, visiting the positions in cell order, but its sort
 * scratch (bins, permutation, bin counters) is one fixed array compiled into the
 * library (about 8.7 MB, held on every GPU that loads the library until the process
 * exits) instead of memory the handle allocates.  The caller still passes the
 * positions and the outputs, laid out as for qmcspl_eval_vgl.
 *   n_pos  0 .. QMCSPL_NOALLOC_MAX_POS; larger counts fail with QMCSPL_ERR_ARG
 *          before anything is launched
 * Bloch handles are not accepted (QMCSPL_ERR_UNSUPPORTED): their phase factors need
 * per-position scratch that the fixed array does not hold.
 *   stream cudaStream_t; asynchronous like qmcspl_eval_vgl
 * The first call on a device looks up the array's device address (a one-time set-up
 * per device, under a lock); make that first call before capturing any stream.
 * Every call on a device shares the one array and leaves its contents behind; each
 * call clears the counters it needs, but calls whose work overlaps on the GPU (on
 * different streams, or from different threads) race on the array and must be
 * ordered by the caller.  qmcspl_profile does not record these calls.
 */
#define QMCSPL_NOALLOC_MAX_POS (1 << 20)
int qmcspl_eval_vgl_noalloc(qmcspl_t h, const double* pos, long long n_pos, void* val,
                            void* grad, void* lap, void* stream);

/*
 * qmcspl_slater_kinetic -- a consumer of the orbital outputs: the Slater matrices of a
 * walker batch, their log-determinants, the local kinetic energy and the drift.
 *
 * Paper, Sec. I: the trial wave function is a Jastrow factor times a Slater determinant of
 * the single-particle orbitals; the local energy is H Psi / Psi.  Here Psi = det A_up det A_dn
 * (no Jastrow factor): for walker w, spin block s with electrons e0 .. e0 + n_s - 1 (e0 = 0,
 * n_s = n_up for spin up; e0 = n_up, n_s = n_elec - n_up for spin down)
 *     A_s[i][j] = val[w n_elec + e0 + i][j],   j < n_s (the first n_s orbitals),
 * and, by Jacobi's formula,
 *     logdet[w]  = ln|det A_up| + ln|det A_dn|,   sign[w] = sign(det A_up det A_dn)
 *     kinetic[w] = -1/2 sum_s tr(A_s^-1 L_s),   L_s[i][j] = lap[w n_elec + e0 + i][j]
 *                  (the kinetic part of the local energy, hartree)
 *     drift[w][e][c] = sum_j (A_s^-1)_ji grad[w n_elec + e][c][j]   (d_c ln|Psi| for electron e)
 * Determinant updates (one electron moved) are not provided.
 *
 *   val, grad, lap  device outputs of qmcspl_eval_vgl for P = n_walkers x n_elec positions
 *          ordered walker-major, layouts [P][n_orb], [P][3][n_orb], [P][n_orb]; dtype 0 = double,
 *          1 = float (real orbitals), 2 = complex double, 3 = complex float (Bloch orbitals,
 *          the (re, im) layouts of a Bloch handle's outputs)
 *   arith  enum qmcspl_slater_arith, for real and complex dtypes
 *   n_orb  the output row length O (orbitals), >= both block sizes
 *   n_up   0 .. n_elec; each block at most QMCSPL_SLATER_MAX_BLOCK electrons
 *          (QMCSPL_SLATER_MAX_COMPLEX_BLOCK for complex dtypes)
 *   logdet device double[n_walkers] or NULL
 *   sign, kinetic  device double[n_walkers] or NULL (kinetic needs lap); for complex dtypes
 *          double[n_walkers][2]: sign = (cos, sin) of the phase of det A_up det A_dn, kinetic
 *          = the complex kinetic term (re, im)
 *   drift  device double[n_walkers][n_elec][3] or NULL (needs grad); complex dtypes
 *          double[n_walkers][n_elec][3][2]
 *   stream cudaStream_t; asynchronous
 * The inversion is Gauss-Jordan elimination with row pivoting in shared memory, one thread
 * block per walker, in FP64 or in double-float (arith); complex entries are pivoted on the
 * largest modulus, and in double-float each of their parts is a float pair.  An exactly
 * singular block gives sign 0, logdet -inf and NaN kinetic energy and drift for that walker;
 * nearly singular blocks lose accuracy as the condition number grows.
 */
#define QMCSPL_SLATER_MAX_BLOCK 160
#define QMCSPL_SLATER_MAX_COMPLEX_BLOCK 112
enum qmcspl_slater_arith {
    QMCSPL_SLATER_FP64 = 0,   /* FP64 elimination (GB300's FP64 pipe) */
    QMCSPL_SLATER_DF64 = 1    /* double-float elimination on the FP32 pipe: each entry a pair
                                 of floats (~48 significant bits), error-free FP32 updates;
                                 results agree with FP64 to about 1e-13 times the condition
                                 number */
};
int qmcspl_slater_kinetic(const void* val, const void* grad, const void* lap, int dtype, int arith,
                          long long n_walkers, int n_elec, int n_up, int n_orb, double* logdet, double* sign,
                          double* kinetic, double* drift, void* stream);

/*
 * qmcspl_debug_fail_alloc -- test hook: make one device allocation of the library fail.
 *
 * Not in the paper.  After n further successful device allocations (any call, any thread)
 * the next one reports cudaErrorMemoryAllocation, as if the device were full; the hook then
 * switches itself off.  n < 0 switches it off.  Every entry point must then return
 * QMCSPL_ERR_OOM (or QMCSPL_ERR_CUDA) and release what it had allocated, leaving the handle
 * (if any) usable.  Returns QMCSPL_OK.
 */
int qmcspl_debug_fail_alloc(long long n);

/*
 * qmcspl_debug_stall_pipeline -- test hook: the next n staged evaluations (pencil order)
 * run with a producer warp that copies nothing, so that every consumer wait of the
 * pipeline runs out (about a second) exactly as it would if the pipeline had stalled.  The
 * launch then ends on its own; qmcspl_sync returns QMCSPL_ERR_TIMEOUT, the outputs of that
 * call are undefined, and the handle stays usable.  n <= 0 switches the hook off.  Returns
 * QMCSPL_OK.
 */
int qmcspl_debug_stall_pipeline(int n);

/*
 * qmcspl_profile / qmcspl_profile_read -- CUDA-event timing of the library's own kernels.
 *
 * Not in the paper.  While enabled, every qmcspl_eval_vgl on the handle records CUDA
 * events on its stream around the cell-ordering kernels and around the evaluation
 * kernel (up to 4096 calls).  qmcspl_profile(h, 1) enables and clears the record,
 * qmcspl_profile(h, 0) disables it.  qmcspl_profile_read synchronises on the recorded
 * events and returns the summed device time in milliseconds of the evaluation
 * kernel launches (eval_ms), of the ordering kernels (order_ms) and the number of
 * evaluation launches recorded.  Any output pointer may be NULL.
 */
int qmcspl_profile(qmcspl_t h, int enable);
int qmcspl_profile_read(qmcspl_t h, double* eval_ms, double* order_ms, long long* launches);

/*
 * qmcspl_save / qmcspl_load -- keep built tables on disk (checkpoint and resume).
 *
 * Not in the paper.  qmcspl_save writes the handle's geometry (lattice, grid, orbital
 * count, method, storage, layout) and its tables, byte for byte, with a 64-bit FNV-1a
 * checksum of the table bytes; it synchronises the device and blocks.  qmcspl_load
 * reads such a file and builds a handle on the current device without the planewave
 * construction (the tables are uploaded as stored, on `stream`; the call blocks).
 * A file that is truncated, carries another magic, format or layout version, has
 * inconsistent sizes or fails the checksum is rejected with QMCSPL_ERR_ARG before any
 * device memory is allocated; I/O failures give QMCSPL_ERR_ARG with the OS message.
 */
int qmcspl_save(qmcspl_t h, const char* path);
int qmcspl_load(qmcspl_t* out, const char* path, void* stream);

/*
 * qmcspl_probe_cache -- measured throughput of the SMs' L1 or L2 data path (not in the paper).
 *
 * Every evaluation gathers 64 coefficient rows per table (Sec. III B).  With positions in
 * cell order most of those rows are shared with neighbouring positions and come from the SMs'
 * L1 caches or from L2, so the rates that bound the evaluation kernels are how fast L1 and L2
 * return 16-byte loads, not the HBM rate.  This call measures one of them on the current
 * device: two 1024-thread blocks per SM issue 16-byte loads shaped like the evaluation
 * kernels' (each warp instruction 512 contiguous bytes), eight independent loads per thread in
 * flight; each launch is timed with CUDA events on `stream`, best of five after one warm-up.
 *   level          1: read-only loads (ld.global.nc) over a 64 KB buffer resident in every L1;
 *                  2: L2-only loads (ld.global.cg) over a 32 MB buffer resident in L2
 *   gbs            [out] bytes returned per second to all SMs together, GB/s
 *   bytes_per_clk  [out] the same per SM and per SM clock cycle
 *   sm_mhz         [out] the SM clock of the best launch (clock64 cycles / event time)
 * Any output may be NULL.  Blocking.  Allocates the buffer (64 KB or 32 MB) for the call and
 * frees it before returning; changes no device setting.  QMCSPL_ERR_ARG for another level.
 */
int qmcspl_probe_cache(int level, double* gbs, double* bytes_per_clk, double* sm_mhz, void* stream);

/*
 * qmcspl_probe_fma -- measured FP32 multiply-add throughput of the SMs (not in the paper).
 *
 * Where positions share their stencil rows on chip, the kernels that also form the Hessian or
 * the pp-spline derivatives spend their time in multiply-adds (z sums and column weights per
 * orbital, Eq. (b-splineapproximation)), and the rate that bounds them is that of the FP32
 * pipe.  This call measures it on the current device: two 1024-thread blocks per SM, each thread
 * eight independent chains of 4096 multiply-adds, timed with CUDA events on `stream`, best of five
 * after one warm-up.
 *   packed         0: fma.rn.f32 (one multiply-add per lane and instruction);
 *                  1: fma.rn.f32x2 (two per lane and instruction, the form the kernels use)
 *   tflops         [out] multiply-add FLOPs per second (2 per multiply-add), 10^12
 *   flops_per_clk  [out] the same per SM and per SM clock cycle
 *   sm_mhz         [out] the SM clock of the best launch (clock64 cycles / event time)
 * Any output may be NULL.  Blocking; allocates a few KB for the call; changes no device
 * setting.  QMCSPL_ERR_ARG for another value of packed.
 */
int qmcspl_probe_fma(int packed, double* tflops, double* flops_per_clk, double* sm_mhz, void* stream);

/* qmcspl_sync -- synchronise `stream` and report (then clear) any device-side error the
 * handle's kernels recorded: QMCSPL_ERR_DEVICE for non-finite positions. */
int qmcspl_sync(qmcspl_t h, void* stream);

/* qmcspl_last_error -- message of the last failed call on this thread ("" if none). */
const char* qmcspl_last_error(void);

/* qmcspl_version -- library version as 10000*major + 100*minor + patch. */
int qmcspl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QMCSPL_H */
