/*
 * dfsnufft -- GB300 (sm_103a) type-2 NUFFT for DFS spectral interpolation.
 *
 * The operation (Sec. 5, Eq. 5.3): given the complex coefficients c_{n,m} of a
 * field's bivariate Fourier series on the doubled sphere and P departure
 * points (phi_p, theta_p), evaluate
 *
 *     v_p = sum_{n=-N2/2}^{N2/2-1} sum_{m=-N1/2}^{N1/2-1} c_{n,m} e^{i m phi_p} e^{i n theta_p}
 *
 * for every point: the type-II nonuniform DFT that the paper evaluates with a
 * NUFFT (Sec. 5) in place of Lagrange interpolation at the semi-Lagrangian
 * departure points (Sec. 2).  For an n_lat x n_lon Grid [0] (Sec. 3,
 * n_lon = 2J) the coefficient array is N2 x N1 = (2 n_lat) x n_lon.
 *
 * Method: exponential-of-semicircle spreading kernel of width w and shape
 * beta = 2.30 w, oversampling sigma >= 2 to power-of-two fine sizes;
 * deconvolve-and-pad, 2-D inverse FFT (sign +1), then a w x w interpolation
 * at each point from the fine grid.  w is the narrowest width whose modelled
 * 1-D interpolation error is at most 2.5 tol (F64) or 5 tol (F32), so that
 * even a lone mode at the corner of the band (the worst band-limited input)
 * stays within half of the accepted relative error, 10 tol (F64) or 20 tol
 * (F32): w = 14 at tol 1e-12, 16 at 1e-14, 7 at 1e-6.
 *
 * Conventions common to every entry point
 *  - Coefficients: n_fields x N2 x N1 complex, C-contiguous, interleaved
 *    (re, im), m fastest.  Row r <-> n = r - N2/2, column q <-> m = q - N1/2.
 *    complex128 for DFSNUFFT_F64 plans, complex64 for DFSNUFFT_F32 plans.
 *    The Nyquist row/column (n = -N2/2, m = -N1/2) are evaluated literally.
 *  - Points: two arrays of n_points float64 (radians): longitude phi and
 *    colatitude theta.  Any real value is accepted; both are wrapped by
 *    2 pi periodicity of the doubled torus.  Points with colatitude in
 *    [0, pi] (the physical sphere) touch only half of the fine grid, and only
 *    that half is computed.
 *  - Values: n_fields x n_points real (float64 or float32 by plan dtype),
 *    Re(v_p) in the caller's point order.
 *  - Streams: every device call is enqueued on the plan's CUDA stream and
 *    returns after enqueue (asynchronous); results are ready when the stream
 *    reaches that point.  A plan is not thread-safe.
 *  - Ownership: the caller allocates and owns every input and output buffer.
 *    The plan owns its fine grids, deconvolution factors, twiddle tables and
 *    sorted point data; set_points copies what it needs, so the point
 *    buffers may be reused once the stream has passed the call.
 *  - Errors: every function returns a status (0 = DFSNUFFT_OK).  No exception
 *    or abort crosses this boundary.  A CUDA failure makes the plan's status
 *    sticky: later calls on that plan return DFSNUFFT_ERR_CUDA until it is
 *    destroyed; dfsnufft_plan_last_error() gives the message.
 */
#ifndef DFSNUFFT_H
#define DFSNUFFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dfsnufft_plan_s *dfsnufft_plan;

/* Arithmetic type of a plan. */
enum { DFSNUFFT_F64 = 0, DFSNUFFT_F32 = 1 };

/* Status codes. */
enum {
    DFSNUFFT_OK = 0,
    DFSNUFFT_ERR_INVALID_ARG = 1,      /* bad size, dtype, null pointer, odd dims   */
    DFSNUFFT_ERR_TOL_UNATTAINABLE = 2, /* tol below 1e-14 (F64) or 1e-7 (F32)       */
    DFSNUFFT_ERR_NO_POINTS = 3,        /* execute before set_points                 */
    DFSNUFFT_ERR_OOM = 4,              /* device allocation failed                  */
    DFSNUFFT_ERR_CUDA = 5,             /* a CUDA call failed (sticky per plan)      */
    DFSNUFFT_ERR_UNSUPPORTED = 6,      /* size outside the supported range          */
    DFSNUFFT_ERR_TIMEOUT = 7           /* a kernel gave up waiting on an async copy */
};

/* Parameters a plan chooses (also available without a GPU). */
typedef struct {
    int n_lon, n_lat;      /* grid: N1 = n_lon phi-modes, N2 = 2 n_lat theta-modes  */
    int N1, N2;            /* coefficient array dims (columns, rows)               */
    int n1, n2;            /* fine (oversampled) grid dims, powers of two          */
    int w;                 /* kernel width in fine-grid cells                      */
    double beta;           /* kernel shape parameter                               */
    double tol;            /* requested tolerance                                  */
    int dtype;             /* DFSNUFFT_F64 or DFSNUFFT_F32                          */
    int tile_x, tile_y;    /* interpolation bin size in fine cells                 */
    int sigma;             /* oversampling factor (2 or 4)                          */
    unsigned flags;        /* DFSNUFFT_REAL_FIELDS | _KEEP_ORDER | _GAUSS_GRID, or 0 */
} dfsnufft_params;

/* ---- plan options -------------------------------------------------------- */

/* The fields are real on the sphere (the SWE fields h, u, v of the paper are),
 * so their coefficients are Hermitian: c_{-n,-m} = conj(c_{n,m}) for every
 * pair of entries that both lie in the array.  The plan then reads only the
 * columns m >= 0, the Nyquist column m = -N1/2 and the Nyquist row
 * n = -N2/2, transforms half of the columns and keeps half of the theta-pass
 * buffer.  The values are Re v for the coefficients whose columns
 * -N1/2 < m < 0 are, off the Nyquist row, the conjugate mirrors of columns -m;
 * every entry of the Nyquist row and column is evaluated literally, as in a
 * general plan.  For Hermitian input this is Re v exactly. */
#define DFSNUFFT_REAL_FIELDS 1u

/* Points are evaluated in the caller's order, without the sort by
 * interpolation bin: set_points only folds them (one pass), and each point's
 * stencil is read from the fine grid through the L1 cache.  Meant for point
 * sets whose consecutive points are close on the sphere, such as the
 * semi-Lagrangian departure points of a latitude-longitude grid in raster
 * order; any order gives the same values (only slower). */
#define DFSNUFFT_KEEP_ORDER 2u

/* The arrival grid's latitudes are the n_lat Gauss-Legendre nodes (Sec. 3, the
 * GL grid; colatitude theta_j = arccos(z_j), increasing from the north pole)
 * instead of Grid [0].  dfsnufft_grid_to_coeffs and dfsnufft_interpolate_grid
 * then take samples on that grid: the FFT in longitude and, in latitude, the
 * inversion of the DFT matrix of the doubled column (Sec. 5, interpolation for
 * the spherical-harmonic model), split by the field parity into two real
 * n_lat x n_lat solves whose inverses the plan forms once in FP64 on the host
 * (plan creation takes O(n_lat^3) host time: about a second at n_lat = 1024)
 * and applies as GEMMs (cuBLAS).  Same size limits as dfsnufft_grid_to_coeffs.
 * dfsnufft_plan_latitudes returns the nodes. */
#define DFSNUFFT_GAUSS_GRID 4u

/* Options of dfsnufft_plan_create_opts.  A zero-filled struct gives the
 * defaults of dfsnufft_plan_create.
 *   flags  : any of DFSNUFFT_REAL_FIELDS, DFSNUFFT_KEEP_ORDER,
 *            DFSNUFFT_GAUSS_GRID (or 0).
 *   sigma  : oversampling factor, 0 (= 2), 2 or 4.  With 4 the fine grid has
 *            4x the cells of sigma 2 and the kernel may be narrower (the width
 *            rule keeps the kernel's modelled interpolation error at or below
 *            that of sigma 2 at the same tol); beta = 0.97 pi (1 - 1/(2 sigma)) w.
 *   w      : kernel width 2..16, 0 = from tol and sigma.  A width below the
 *            rule's lowers the accuracy (the autotuner checks it).
 *   tile_x, tile_y : interpolation bin in fine cells, powers of two from 8 to
 *            128 (0 = the default: 32 x 16 for F32, 128 x 16 for F64); tile_y is
 *            raised to n2/512 when smaller. */
typedef struct {
    unsigned flags;
    int sigma;
    int w;
    int tile_x, tile_y;
} dfsnufft_options;

/* Parameters with options (opts may be NULL for the defaults). */
int dfsnufft_choose_params_opts(int n_lon, int n_lat, double tol, int dtype,
                                const dfsnufft_options *opts, dfsnufft_params *out);

/* Create a plan for an n_lat x n_lon grid.
 *   n_lon : even, >= 4; N1 = n_lon phi-modes.  n_lat >= 2; N2 = 2 n_lat.
 *   tol   : requested relative accuracy, 1e-14 <= tol < 1 (F64),
 *           1e-7 <= tol < 1 (F32).
 *   dtype : DFSNUFFT_F64 or DFSNUFFT_F32.
 *   n_fields : fields evaluated per execute at the same points (>= 1).
 *   stream : cudaStream_t to enqueue on (NULL = legacy default stream).
 *   out    : receives the plan handle (owned by the library until destroy).
 * Fine grids up to 8192 x 8192 are supported (ERR_UNSUPPORTED above). */
int dfsnufft_plan_create(int n_lon, int n_lat, double tol, int dtype, int n_fields,
                         void *stream, dfsnufft_plan *out);

/* A batched plan (n_members >= 1, see dfsnufft_plan_create_batch) with
 * options (opts may be NULL: the defaults). */
int dfsnufft_plan_create_opts(int n_members, int n_lon, int n_lat, double tol, int dtype,
                              int n_fields, const dfsnufft_options *opts, void *stream,
                              dfsnufft_plan *out);

/* Give a one-member plan its departure points (device pointers, float64
 * radians, n_points each, 1 <= n_points < 2^31).  Folds them onto the
 * fine-grid torus (exact integer reduction of the angles), sorts them by
 * interpolation bin (counting sort) and finds the fine rows their stencils
 * touch.  Replaces any previous points. */
int dfsnufft_set_points(dfsnufft_plan plan, int64_t n_points, const double *lon,
                        const double *colat);

/* Batched plans: n_members members on the same n_lat x n_lon grid, each with
 * its own departure points and n_fields fields (an ensemble, or several
 * requests of one size).  Arguments as dfsnufft_plan_create; 1 <= n_members
 * <= 4096 and n_members x n_fields <= 65535.  A plan from dfsnufft_plan_create is a batched plan of one member.
 * Member data are concatenated in member order:
 *   coeffs : n_members x n_fields x N2 x N1 complex,
 *   points : all members' longitudes (then colatitudes) back to back,
 *   values : for member k, n_fields x n_points[k] reals, members back to back. */
int dfsnufft_plan_create_batch(int n_members, int n_lon, int n_lat, double tol, int dtype,
                               int n_fields, void *stream, dfsnufft_plan *out);

/* Points of every member of a batched plan: n_points is a host array of
 * n_members counts (each >= 1, total < 2^31); lon and colat are device arrays
 * of the total length, member k's points at offset sum_{j<k} n_points[j].
 * The offsets are uploaded (a small host-to-device copy on the plan's stream)
 * only when the counts differ from the previous call's. */
int dfsnufft_set_points_batch(dfsnufft_plan plan, const int64_t *n_points, const double *lon,
                              const double *colat);

/* Ensembles on uneven grids: n_groups batched plans (group g: n_members[g]
 * members on an n_lat[g] x n_lon[g] grid, all with n_fields fields, one
 * tolerance and precision), each on a stream of its own. */
typedef struct dfsnufft_ensemble_s *dfsnufft_ensemble;
int dfsnufft_ensemble_create(int n_groups, const int *n_members, const int *n_lon,
                             const int *n_lat, double tol, int dtype, int n_fields, void *stream,
                             dfsnufft_ensemble *out);

/* The same with per-group plan options: opts is NULL (defaults) or an array of
 * n_groups options (for instance the autotuner's choice per grid size). */
int dfsnufft_ensemble_create_opts(int n_groups, const int *n_members, const int *n_lon,
                                  const int *n_lat, double tol, int dtype, int n_fields,
                                  const dfsnufft_options *opts, void *stream,
                                  dfsnufft_ensemble *out);

/* One step for every member of every group: per group g, n_points[g] (host
 * array of the group's member counts), lon[g], colat[g], coeffs[g], values[g]
 * (device pointers laid out as for dfsnufft_set_points_batch and
 * dfsnufft_execute).  The step is recorded as one CUDA graph (a fork over the
 * group streams and a join back into the ensemble's stream) and replayed with
 * one graph launch on later calls with the same pointers and counts; a call
 * with other pointers or counts runs the step once as is and records it anew.
 * Asynchronous on the ensemble's stream. */
int dfsnufft_ensemble_run(dfsnufft_ensemble ens, const int64_t *const *n_points,
                          const double *const *lon, const double *const *colat,
                          const void *const *coeffs, void *const *values);

/* Synchronise and report the first failure of any group (DFSNUFFT_OK if none). */
int dfsnufft_ensemble_check(dfsnufft_ensemble ens);

/* The batched plan of group g (owned by the ensemble). */
int dfsnufft_ensemble_plan(dfsnufft_ensemble ens, int group, dfsnufft_plan *out);

/* Persistent mode (on = 1) or the fork/join graph (on = 0, the default) for the
 * next steps.  In persistent mode each group's set_points still runs as a branch
 * of the step's graph, and the theta pass, phi pass and interpolation of every
 * member of every group then run as ONE persistent launch, recorded in the same
 * graph: its CTAs drain a device work queue that lists all groups' theta tasks
 * (column blocks), then their phi tasks (row blocks), then their interpolation
 * tasks (bins); a phi task waits until its group's theta tasks are done and an
 * interpolation task until its group's phi tasks are done (Sec. 5, the NUFFT of
 * Eq. 5.3 for many fields and members of uneven grids at once).  Each wait is
 * bounded (about a second); one that runs out ends the launch early and
 * dfsnufft_ensemble_check then returns DFSNUFFT_ERR_TIMEOUT.  Supported for
 * FP32 ensembles of at most 16 groups whose plans keep points sorted, have
 * kernel width 6 or 7 and fine grids from 256 to 4096 cells a side; otherwise
 * DFSNUFFT_ERR_UNSUPPORTED and the mode is unchanged.  The step is recorded
 * again on the next run. */
int dfsnufft_ensemble_set_persistent(dfsnufft_ensemble ens, int on);

int dfsnufft_ensemble_destroy(dfsnufft_ensemble ens);

/* ---- serving: continuous batching under an HBM budget ------------------- */

/* One member's interpolation step: its grid, n_points departure points and
 * n_fields coefficient arrays (device pointers, layouts as for a one-member
 * plan), and a device buffer of n_fields x n_points values to fill.  The
 * buffers must stay valid until the request completes. */
typedef struct {
    int n_lon, n_lat;
    int64_t n_points;
    const double *lon;
    const double *colat;
    const void *coeffs;
    void *values;
} dfsnufft_request;

typedef struct {
    int64_t submitted, completed;   /* requests                                   */
    int64_t batches, members;       /* batched launches and requests they carried */
    int slots;                      /* live slots (stream + batched plan + staging) */
    int64_t reserved_bytes;         /* device bytes the slots hold                */
    int64_t budget_bytes;           /* the HBM budget                             */
} dfsnufft_server_stats;

typedef struct dfsnufft_server_s *dfsnufft_server;

/* A server for requests of any grid at tolerance tol, precision dtype, with
 * n_fields fields each.  A dispatcher thread groups queued requests by grid and
 * launches up to max_batch of one grid as one batched plan execution on a free
 * slot; slots are created while the device memory they need fits hbm_budget
 * (bytes) and are kept for reuse.  Requests arriving while others run are
 * admitted as soon as a slot frees up, so their work overlaps on the device.
 * Uses the device current at creation. */
int dfsnufft_server_create(double tol, int dtype, int n_fields, int64_t hbm_budget,
                           int max_batch, dfsnufft_server *out);

/* The same with plan options for every slot (opts may be NULL; tile sizes
 * that do not fit a grid are clamped as for a plan). */
int dfsnufft_server_create_opts(double tol, int dtype, int n_fields, int64_t hbm_budget,
                                int max_batch, const dfsnufft_options *opts,
                                dfsnufft_server *out);

/* Queue a request (thread-safe; returns at once with a ticket). */
int dfsnufft_server_submit(dfsnufft_server srv, const dfsnufft_request *req, int64_t *ticket);

/* Wait up to timeout_s seconds for a ticket: *status is the request's outcome
 * (DFSNUFFT_OK, or DFSNUFFT_ERR_OOM when no slot for its grid can ever fit the
 * budget, or a CUDA error), *latency_s the time from submit to completion.
 * Returns DFSNUFFT_ERR_TIMEOUT if the request is still running. */
int dfsnufft_server_wait(dfsnufft_server srv, int64_t ticket, double timeout_s, int *status,
                         double *latency_s);

int dfsnufft_server_stats_get(dfsnufft_server srv, dfsnufft_server_stats *out);

/* Finish queued and running requests, then release every slot. */
int dfsnufft_server_destroy(dfsnufft_server srv);

/* Evaluate all n_fields series at the plan's points (Eq. 5.3).
 *   coeffs : device pointer, (n_members x) n_fields x N2 x N1 complex (see conventions).
 *   values : device pointer, (members back to back) n_fields x n_points real,
 *            written in full. */
int dfsnufft_execute(dfsnufft_plan plan, const void *coeffs, void *values);

/* Evaluate fields given by the coefficients of the paper's partial-regularity
 * DFS expansion (Sec. 4):
 *   f = sum_m F^c_m(theta) cos m phi + F^s_m(theta) sin m phi,
 *   F_0 = sum_{n=0}^{N} f_{n,0} cos n theta,
 *   F_1 = sum_{n=0}^{N-1} f_{n,1} sin theta cos n theta,
 *   F_m = sum_{n=1}^{N-1} f_{n,m} sin theta sin n theta      (even m >= 2),
 *   F_m = sum_{n=1}^{N-2} f_{n,m} sin^2 theta sin n theta    (odd m >= 3),
 * at the plan's points.  The coefficients are converted to the complex ones of
 * Eq. 5.4 inside the theta pass (through the standard DFS coefficients, Sec. 4),
 * with no extra pass over memory.
 *   pr : device pointer, (n_members x) n_fields x (M + 1) x (N + 1) complex in
 *        plan precision, element [m][n] = f^c_{n,m} + i f^s_{n,m} (n fastest);
 *        entries outside each m's index range above, and the sine part of
 *        m = 0, are ignored.
 *   0 <= M <= n_lon/2 - 1, 1 <= N <= n_lat - 1.  The plan must be a real-field
 *   plan (DFSNUFFT_REAL_FIELDS); values as for dfsnufft_execute. */
int dfsnufft_execute_pr(dfsnufft_plan plan, int M, int N, const void *pr, void *values);

/* Coefficients from samples on the arrival grid (Sec. 3-4): samples of every
 * field on Grid [0], theta_j = (j + 1/2) pi / n_lat, phi_k = 2 pi k / n_lon,
 * (members x) n_fields x n_lat x n_lon reals in plan precision (device,
 * phi fastest); parity is a host array of n_fields values, +1 for a scalar
 * field and -1 for a wind component, by which the samples are extended to the
 * doubled sphere (f(phi + pi, -theta) = parity f(phi, theta)).  Writes the
 * centred coefficients of the trigonometric interpolant on the doubled torus,
 *   c_{n,m} = (1 / (N1 N2)) sum_{j,k} f_ext(phi_k, theta_j) e^{-i (m phi_k + n theta_j)},
 * in the layout dfsnufft_execute reads.  Needs n_lon and 2 n_lat powers of two
 * from 16 to 4096 and n_lat even (else DFSNUFFT_ERR_UNSUPPORTED); uses the
 * plan's theta-pass buffer as scratch (stream-ordered, so it may be followed by
 * execute).  A changed parity array is uploaded with a synchronising copy. */
int dfsnufft_grid_to_coeffs(dfsnufft_plan plan, const void *samples, const int *parity,
                            void *coeffs);

/* The arrival grid's colatitudes (n_lat doubles, host): the Gauss-Legendre
 * nodes of a DFSNUFFT_GAUSS_GRID plan, else Grid [0]'s (j + 1/2) pi / n_lat. */
int dfsnufft_plan_latitudes(dfsnufft_plan plan, double *colat);

/* One semi-Lagrangian interpolation step: samples on the arrival grid (as for
 * dfsnufft_grid_to_coeffs) to values at the plan's points (as for
 * dfsnufft_execute), through a plan-owned coefficient buffer. */
int dfsnufft_interpolate_grid(dfsnufft_plan plan, const void *samples, const int *parity,
                              void *values);

/* ---- departure points and the vector rotation (Sec. 2) -------------------- */

/* Departure points of the semi-Lagrangian step, Eq. 2.4 of Sec. 2,
 *   x_D = x - dt [ W(x_D) - W_A(x) ],
 * solved by fixed-point iteration for every arrival point of Grid [0]
 * (theta_j = (j + 1/2) pi / n_lat, phi_k = 2 pi k / n_lon), with W(x_D)
 * carried to the arrival point's frame by the rotation Q of Sec. 2 and the
 * displacement taken along the great circle through the arrival point:
 *   D_0 = A;  V_k = Q(A, D_k) W(D_k) - W_A(A);
 *   D_{k+1} = the point at angle |V_k| dt / a from A in the direction -V_k.
 * W(D) is tensor-product quintic Lagrange interpolation of the samples of W
 * (the degree the paper uses for this bracket), stencil rows beyond a pole
 * taken from the doubled sphere with the wind components' change of sign.
 *   w         : device, n_members x 2 x n_lat x n_lon (eastward, then
 *               northward component; phi fastest), dtype reals: the bracket's
 *               departure term, (v + Omega x r - g dt grad h^(+) / 4) in Eq. 2.4.
 *   w_arrival : same layout, the arrival term (Omega x r + g dt grad h^0 / 4),
 *               or NULL for zero.
 *   dt_over_a : time step divided by the sphere's radius, in the units that
 *               make |W| dt_over_a an angle in radians.
 *   iterations: 1..64 evaluations of W (the first one at the grid point).
 *   lon_d, colat_d: device outputs, n_members x n_lat x n_lon doubles, in grid
 *               order; longitude in [0, 2 pi), colatitude in [0, pi] up to
 *               rounding.  FP32 runs the iteration in single precision
 *               relative to the arrival point (error about 1e-6 of the
 *               displacement); positions are always written in FP64.
 *   pq        : optional device output (NULL to skip), n_members x 2 x
 *               n_lat x n_lon dtype reals: p, then q, of the rotation Q from
 *               each final departure point to its arrival point, for
 *               dfsnufft_rotate_to_arrival.
 * n_lon even >= 6, n_lat >= 3; stream is a cudaStream_t (NULL = legacy
 * default).  Asynchronous; returns DFSNUFFT_ERR_INVALID_ARG or
 * DFSNUFFT_ERR_CUDA (launch failure) without touching any plan. */
int dfsnufft_departure_points(int n_lon, int n_lat, int n_members, int dtype, int iterations,
                              double dt_over_a, const void *w, const void *w_arrival,
                              double *lon_d, double *colat_d, void *pq, void *stream);

/* Vector values at departure points expressed in the arrival points' frame
 * (Sec. 2): (u_a, v_a) = Q (u_d, v_d), Q = [[p, q], [-q, p]] with
 *   p = (sin th_A sin th_D + (1 + cos th_A cos th_D) cos(ph_A - ph_D)) / (1 + cos eta),
 *   q = (cos th_A + cos th_D) sin(ph_A - ph_D) / (1 + cos eta),
 * for the arrival points of Grid [0] in grid order and the departure points
 * (lon_d, colat_d) (device doubles, n_members x n_lat x n_lon), or read from pq
 * as written by dfsnufft_departure_points (then lon_d and colat_d may be NULL;
 * no trigonometry and no FP64 arithmetic, which on this GPU runs at 1/64 of the
 * FP32 rate).  u_d, v_d, u_a,
 * v_a: device dtype reals, point p of member m at [m * stride + p] (stride >=
 * n_lat n_lon; with the values of dfsnufft_execute, stride = n_fields times the
 * points and u_d, v_d the two wind fields).  In place (u_a = u_d, v_a = v_d) is
 * allowed.  Asynchronous on stream; errors as dfsnufft_departure_points. */
int dfsnufft_rotate_to_arrival(int n_lon, int n_lat, int n_members, int dtype,
                               const double *lon_d, const double *colat_d, const void *pq,
                               const void *u_d, const void *v_d, int64_t stride, void *u_a,
                               void *v_a, void *stream);

/* ---- Lagrange interpolation comparator ----------------------------------- */

/* Tensor-product Lagrange interpolation of degree order (3 = cubic, 5 =
 * quintic) of samples on Grid [0] at arbitrary points: the interpolation of the
 * paper's baseline model (cubic for the scalar forcing, quintic for the vector
 * one; Sec. 1-2), for comparison with the spectral path.  Stencil: the
 * (order + 1)^2 grid nodes around the point in index space x = phi n_lon /
 * (2 pi), y = theta n_lat / pi - 1/2; rows beyond a pole and points with a
 * negative colatitude use the doubled sphere, f(phi + pi, -theta) =
 * parity f(phi, theta).
 *   parity : host array of n_fields values, +1 scalar, -1 wind component.
 *   samples: device, n_fields x n_lat x n_lon dtype reals (phi fastest).
 *   lon, colat: device doubles, n_points each, any real value below 2^53 rad
 *            in magnitude, reduced exactly (others give NaN values).
 *   values : device, n_fields x n_points dtype reals.
 * n_lon even and > order, n_lat >= (order + 1) / 2, 1 <= n_fields <= 32.
 * Asynchronous on stream; returns DFSNUFFT_ERR_INVALID_ARG or
 * DFSNUFFT_ERR_CUDA (launch failure). */
int dfsnufft_lagrange_interp(int n_lon, int n_lat, int n_fields, const int *parity, int order,
                             int dtype, int64_t n_points, const double *lon, const double *colat,
                             const void *samples, void *values, void *stream);

/* Host-buffer variants: the same operations with host pointers.  The data are
 * copied to plan-owned device buffers on the plan's stream (pinned host memory
 * makes the copies asynchronous); dfsnufft_execute_host waits for the stream
 * before it returns, so values are ready on return.  coeffs has the layout of
 * dfsnufft_execute; a real-field plan (DFSNUFFT_REAL_FIELDS) copies only the part
 * its theta pass reads: the columns m >= 0, the Nyquist column m = -N1/2 and
 * the Nyquist row n = -N2/2 of every line (the rest must still be allocated).
 * dfsnufft_execute_host copies the coefficients on a stream of the plan's own,
 * after the plan's earlier reads of its staging buffer but not after the other
 * work queued on the plan's stream (such as the set_points before it, which
 * the copy overlaps): the host array must hold its values when the call is
 * made. */
int dfsnufft_set_points_host(dfsnufft_plan plan, int64_t n_points, const double *lon,
                             const double *colat);
int dfsnufft_execute_host(dfsnufft_plan plan, const void *coeffs, void *values);

/* dfsnufft_set_points_host followed by dfsnufft_execute_host (Sec. 5, Eq. 5.3:
 * the values of the fields' series at new points), the two scheduled together:
 * one step of the semi-Lagrangian scheme from host arrays.  Arguments, layouts
 * and results as for those two calls (lon, colat: n_points FP64 each; coeffs,
 * values: the layouts of dfsnufft_execute, plan precision), and as they do it
 * leaves the points set for later execute calls.  For a one-member FP32 plan of
 * two or more fields the copies to the device run in the order field 0's
 * coefficients, points, the other fields' coefficients, so that field 0's theta
 * and phi passes (over every fine row: the range the points need is not known
 * before they are sorted) overlap the copy of the points; each field's values
 * go back as soon as it is done.  Other plans run the two calls in turn.  The
 * copies start after all work queued on the plan's stream before the call; the
 * call waits for the stream before it returns, so the host arrays are free again
 * on return.  Errors: DFSNUFFT_ERR_INVALID_ARG (null pointer, n_points outside
 * [1, 2^31 - 1], a batched plan), DFSNUFFT_ERR_OOM, CUDA failures (sticky). */
int dfsnufft_execute_points_host(dfsnufft_plan plan, int64_t n_points, const double *lon,
                                 const double *colat, const void *coeffs, void *values);

/* Release every device buffer of the plan (synchronises its stream first). */
int dfsnufft_destroy(dfsnufft_plan plan);

/* Static description of a status code. */
const char *dfsnufft_strerror(int status);

/* Last error message recorded on the plan ("" if none). */
const char *dfsnufft_plan_last_error(dfsnufft_plan plan);

/* Synchronise the plan's stream and read its device status word.  Kernels that
 * wait on asynchronous (TMA) copies give up after about one second and record
 * a timeout there instead of hanging; this call then returns
 * DFSNUFFT_ERR_TIMEOUT (sticky for the plan).  Otherwise it returns the plan's
 * status (DFSNUFFT_OK when healthy). */
int dfsnufft_plan_check(dfsnufft_plan plan);

/* Parameters of an existing plan. */
int dfsnufft_plan_get_params(dfsnufft_plan plan, dfsnufft_params *out);

/* Stage timing.  Stages: 0 set_points (fold, scan, scatter), 1 theta pass
 * (deconvolve, pad, column FFTs), 2 phi pass (row FFTs), 3 interpolation.
 * When enabled, the plan records a CUDA event pair around every stage on its
 * stream.  dfsnufft_plan_read_timing synchronises the stream, adds the elapsed
 * times of all pending pairs to the running totals, and copies the totals
 * (milliseconds) and the number of timed calls of each stage into the
 * caller's arrays of DFSNUFFT_N_STAGES entries; enabling resets the totals.
 * Measurement aid of this library; the paper has no counterpart. */
#define DFSNUFFT_N_STAGES 4
int dfsnufft_plan_enable_timing(dfsnufft_plan plan, int enable);
int dfsnufft_plan_read_timing(dfsnufft_plan plan, double *ms_total, int64_t *calls);

/* Work statistics of the current points (synchronises the stream): the
 * number of fine rows computed per field (one circular range, in blocks of 16
 * rows, covering every row the points' stencils touch) and the number of
 * non-empty interpolation bins.  Measurement aid; no paper counterpart. */
int dfsnufft_plan_point_stats(dfsnufft_plan plan, int64_t *rows_needed, int64_t *nonempty_bins);

/* Bytes the host-buffer variants move per call at the plan's current points:
 * host to device by dfsnufft_set_points_host (points) and by
 * dfsnufft_execute_host (coefficients), device to host by dfsnufft_execute_host
 * (values).  Measurement aid; no paper counterpart.  DFSNUFFT_ERR_INVALID_ARG
 * for a null pointer. */
int dfsnufft_plan_host_copy_bytes(dfsnufft_plan plan, int64_t *points_h2d, int64_t *coeffs_h2d,
                                  int64_t *values_d2h);

/* ---- autotuner -------------------------------------------------------------- */

/* One workload to tune for (device pointers laid out as for a batched plan's
 * set_points_batch and execute; the buffers are only read). */
typedef struct {
    int n_members, n_lon, n_lat;
    double tol;
    int dtype, n_fields;
    unsigned flags;              /* DFSNUFFT_* option flags: kept by every candidate   */
    const int64_t *n_points;     /* host: n_members point counts                      */
    const double *lon, *colat;   /* device: all members' points                        */
    const void *coeffs;          /* device: n_members x n_fields x N2 x N1, plan type   */
    int steps;                   /* timed steps per candidate (0: 5)                   */
    void *stream;                /* cudaStream_t                                       */
} dfsnufft_tune_args;

typedef struct {
    dfsnufft_options opts;       /* the candidate                                      */
    dfsnufft_params prm;         /* the parameters its plan chose                      */
    double ms;                   /* median time of set_points + execute (ms)           */
    double err;                  /* largest relative l-inf error over the fields at a
                                    sample of member 0's points (up to 4096), against an
                                    FP64 plan at tol 1e-14                             */
    int status;                  /* DFSNUFFT_OK, or why the candidate did not run      */
} dfsnufft_tune_result;

/* Choose the interpolation bin size, the oversampling factor and the kernel
 * width for this workload by timing real plans on it (CUDA events on the given
 * stream; synchronises it).  Stage 1 times every bin size of the candidate set
 * (tile_x in 16..128, tile_y in 8..64, 128 to 4096 cells) at the width rule's
 * kernel and oversampling 2; stage 2 tries, at the fastest bin, one kernel
 * narrower than the rule and oversampling 4 (its own rule and one narrower).
 * A candidate is accepted when its error is at most 10 tol (F64) or 20 tol
 * (F32); *best receives the fastest accepted one (the default configuration is
 * always a candidate).  Up to max_results candidates are copied to results
 * (may be NULL) and their number to *n_results.  Allocates device memory for
 * the reference and one candidate plan at a time.  No paper counterpart: the
 * paper fixes its parameters by hand. */
int dfsnufft_autotune(const dfsnufft_tune_args *args, dfsnufft_tune_result *results,
                      int max_results, int *n_results, dfsnufft_options *best);

/* ---- allocation-free one-shot call -------------------------------------- */

/* Bytes of the library's static device scratch used by dfsnufft_execute_noalloc. */
#define DFSNUFFT_NOALLOC_SCRATCH_BYTES (64u << 20)

/* One-shot evaluation (the work of set_points followed by execute) that
 * allocates no device memory: for callers that cannot call cudaMalloc, such as
 * a model time step that runs inside another framework's memory pool, or a
 * latency-critical loop that must not take the device-wide synchronisation
 * that cudaMalloc/cudaFree imply.  The paper has no counterpart; this is an
 * interface of this library.
 *
 * All working memory (fine grids, theta-pass buffer, kernel tables, bins and
 * sorted points) lives in one static device array of
 * DFSNUFFT_NOALLOC_SCRATCH_BYTES that every GPU which loads this library's
 * module holds until the process exits (under CUDA's default lazy module
 * loading, from the first call on that GPU).  Arguments are those of dfsnufft_plan_create,
 * dfsnufft_set_points and dfsnufft_execute (device pointers; the caller owns
 * inputs and outputs), with stream = cudaStream_t (NULL = legacy default).
 *   - A problem whose working memory exceeds the scratch, or whose fine grid
 *     exceeds 2048 cells in a dimension, is rejected with
 *     DFSNUFFT_ERR_UNSUPPORTED before anything is enqueued.
 *   - The first call on a device resolves the scratch's device address
 *     (cudaGetSymbolAddress, which may load the module); make that first call
 *     before any stream capture on that device.
 *   - Every call on a device shares the same scratch, which keeps the last
 *     call's contents.  Each call first rewrites what it reads there (its point
 *     offsets, deconvolution factors and twiddles, by one small kernel whose
 *     arguments carry them; counters are cleared before counting), so no
 *     result depends on an earlier call, and no host memory is read after the
 *     call returns.  Calls that overlap on the GPU (other streams, other host
 *     threads) race on the scratch: order them on one stream or synchronise
 *     between them. */
int dfsnufft_execute_noalloc(int n_lon, int n_lat, double tol, int dtype, int n_fields,
                             int64_t n_points, const double *lon, const double *colat,
                             const void *coeffs, void *values, void *stream);

/* ---- host-only helpers (no GPU needed) ---------------------------------- */

/* Parameters a plan with these arguments would use. */
int dfsnufft_choose_params(int n_lon, int n_lat, double tol, int dtype, dfsnufft_params *out);

/* The kernel phi(z) = exp(beta (sqrt(1 - (2z/w)^2) - 1)) for |z| < w/2, else 0
 * (z in fine-grid cells). */
double dfsnufft_es_kernel(double z, int w, double beta);

/* Fourier transform of the kernel at the centred modes of a length-n_modes
 * series on a fine grid of n_fine cells:
 *   out[q] = integral phi(z) cos(2 pi k z / n_fine) dz,  k = q - n_modes/2,
 * by Gauss-Legendre quadrature in FP64.  Deconvolution divides by these. */
int dfsnufft_kernel_ft(int w, double beta, int n_fine, int n_modes, double *out);

/* Piecewise-polynomial form of the kernel used by the interpolation kernels:
 * for tap a (0 <= a < w) the weight phi((a - c0) - t) as a polynomial of degree
 * w in s = t - mid, where t is the point's offset from its base cell
 * (t in [-1/2, 1/2), mid = 0, for odd w; t in [0, 1), mid = 1/2, for even w)
 * and c0 = (w - 1)/2 or w/2 - 1.  out[a * (w + 1) + k] is the coefficient of
 * s^k, from Chebyshev interpolation at w + 1 nodes (FP64).  The fit is
 * accurate to about e^-beta, the size of the kernel's own jump at the edge of
 * its support. */
int dfsnufft_es_horner(int w, double beta, double *out);

/* Library version string. */
const char *dfsnufft_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DFSNUFFT_H */
