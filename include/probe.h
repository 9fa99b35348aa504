/*
 * probe.h -- C ABI of the GB300 matrix-probing library.
 *
 * The library applies the wave-equation normal operator H = F*F to batches of
 * model-space trial functions and fits/applies a pseudodifferential
 * approximation of its inverse, following Demanet et al., "Matrix probing: a
 * randomized preconditioner for the wave-equation Hessian":
 *   - F   Born (linearised) modelling: m0 du_tt - Lap du = -dm (u0)_tt with
 *         m0 (u0)_tt - Lap u0 = delta(x - s) w(t), data = du at the receivers
 *         (Sec. 2, the two wave equations and the definition of d(r,s,t));
 *   - F*  its exact discrete adjoint, reverse-time migration with the zero-lag
 *         imaging condition (Sec. 1.1, "most accurately computed by
 *         reverse-time migration");
 *   - H   = F*F stacked over sources (Sec. 1.1, H = F*F; Sec. 2, the stack
 *         over sources);
 *   - fit the randomized least-squares fit of the coefficients c_i of
 *         H^{-1} = sum_i c_i B_i (Sec. 1.4, Eq. expand and the normal
 *         equations M c = (Bx)^T y), with B_i the elementary operators of
 *         Eq. compr2 (Sec. 1.2);
 *   - precond  sum_i c_i B_i applied to an image (end of Sec. 1.5).
 *
 * Discretisation: 2nd order in time, 8th order in space, on the stated grid
 * (the "interior") surrounded by an absorbing sponge of `pad` cells on every
 * side; the Laplacian is zero-extended beyond the padded grid.  With
 * s = dt^2/m0 and a+- = 1 +- eta dt/2 (eta the sponge damping, zero inside):
 *     u^{n+1} = [2u^n - a- u^{n-1} + s (L u^n + f^n)] / a+ ,  u^{-1} = u^0 = 0,
 * f^n = w[n] / (h_0 ... h_{d-1}) at the source node, data d^n = R du^n for
 * n = 0..nt-1 (R = point sampling at receiver nodes).
 *
 * Conventions
 *   - Arrays are C order with the depth axis first: a 2D model-space array is
 *     [nz][nx], a 3D one [nz][ny][nx]; index tuples are (iz, ix) / (iz, iy, ix)
 *     into the interior grid.  Model-space vectors live on the interior only.
 *   - Data arrays are [nb][ns][nt][nr] (receivers fastest).
 *   - Every array argument may be host or device memory; the library detects
 *     which (cudaPointerGetAttributes).  The caller owns all I/O buffers.  The
 *     library owns its workspaces, wavefield checkpoints and captured graphs.
 *   - Calls enqueue work on `stream` (a cudaStream_t; NULL = legacy default
 *     stream).  If any array argument is host memory, or finiteness checking
 *     is on (the default), the call synchronises `stream` before returning.
 *   - No exception crosses the ABI.  Every failure returns a probe_status and
 *     leaves a message retrievable with probe_last_error(); on failure the
 *     contents of output buffers are unspecified.
 *   - A handle is not thread-safe: serialise calls on one handle.
 */
#ifndef PROBE_H
#define PROBE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct probe_s* probe_t;              /* opaque, library-owned */
typedef struct CUstream_st* probe_stream_t;   /* identical to cudaStream_t */

typedef enum {
    PROBE_OK = 0,
    PROBE_ERR_ARG = -1,        /* invalid argument (sizes, indices, CFL, pointers) */
    PROBE_ERR_CUDA = -2,       /* a CUDA runtime / cuFFT call failed */
    PROBE_ERR_OOM = -3,        /* device allocation failed */
    PROBE_ERR_TIMEOUT = -4,    /* a bounded device-side wait gave up */
    PROBE_ERR_NONFINITE = -5,  /* NaN or Inf found in an input or an output */
    PROBE_ERR_STATE = -6       /* call not valid in the handle's current state */
} probe_status;

enum { PROBE_SNAP_FP32 = 0, PROBE_SNAP_BF16 = 1, PROBE_SNAP_FP16 = 2 };

/* Grid and numerical options (read once by probe_create). */
typedef struct {
    int ndim;            /* 2 or 3 */
    int n[3];            /* interior size, slowest axis first: {nz, nx} or {nz, ny, nx} */
    double h[3];         /* grid spacing [m], same order */
    int pad;             /* absorbing-sponge width in cells, added on every side (>= 0) */
    int snapshot_dtype;  /* PROBE_SNAP_*: storage type of incident-field checkpoints */
    int kahan;           /* 1: Kahan-compensated FP32 imaging accumulation, 0: plain FP32 */
    int ckpt_stride;     /* steps between checkpoints; 0 = ceil(sqrt(nt)) */
} probe_grid;

/* Description of the elementary operators B_i of the symbol expansion
 * (Eq. compr2; 3D uses spherical harmonics in angle, Sec. 1.2).  Term
 * i = (lam * nangular + a) * nradial + q has the symbol
 *     alpha_lam(x) * A_a(k/|k|) * T_q((|k| - L) / (|k| + L)) * |k|^order
 * with T_q the Chebyshev polynomial (TL_q are rational Chebyshev functions),
 * and is applied as B_i x = alpha_lam * IFFT[A_a T_q |k|^order FFT(x)] on the
 * interior zero-padded by fft_pad cells per side; the k = 0 coefficient maps
 * to zero.  Real bases: per-axis spatial factor of mode index k on an axis of
 * n interior cells is 1 (k = 0), cos(2 pi k i / n) (k > 0), sin(2 pi |k| i / n)
 * (k < 0).  2D angular index q: 1 (q = 0), cos(q theta) (q > 0), sin(|q| theta)
 * (q < 0), theta = atan2(k_z, k_x).  3D angular index 0..5: 1, kx ky, ky kz,
 * kx kz, kx^2 - ky^2, 3 kz^2 - 1 of the unit wave vector.  Wave numbers are in
 * rad/m. */
typedef struct {
    int ndim;
    int nspatial;
    const int* spatial;  /* [nspatial][ndim] mode indices, host memory */
    int nangular;
    const int* angular;  /* [nangular], host memory */
    int nradial;
    double L;            /* rational-Chebyshev map scale [rad/m], > 0 */
    double order;        /* exponent of |k| (-1 for the inverse Hessian, Eq. type10_b) */
    int fft_pad;         /* >= 0 */
} probe_basis;

/* Tunables (probe_set_option).  Defaults are chosen by the library. */
typedef enum {
    PROBE_OPT_CHECK_FINITE = 1,  /* 1 (default): check inputs/outputs for NaN/Inf, sync */
    PROBE_OPT_SHOT_WAVE = 2,     /* max shots resident at once; 0 (default) = memory planner */
    PROBE_OPT_SHOT_GROUP = 3,    /* 2D: shots per CTA in the adjoint sweep; 3D: shots per adjoint cluster
                                    (PROBE_OPT_CLUSTER3D bit 1); 0 = autotuned (2D) or 4 (3D) */
    PROBE_OPT_USE_GRAPH = 4,     /* 1 (default): replay sweeps from a captured CUDA graph */
    PROBE_OPT_TIMING = 5,        /* CUDA-event timings read by probe_get_stats (recorded on the call's
                                    stream, also inside replayed graphs; no call synchronises):
                                    1 = every sweep (forward, recompute, adjoint), 2 = the forward
                                    sweep only (two events per shot wave); 0 = off */
    PROBE_OPT_TILE_Z = 6,        /* 2D tile height override (16 or 32); 0 = default */
    PROBE_OPT_PIPELINE = 7,      /* 2D: 0 = one tile per CTA; 2 or 3 = persistent warp-specialised
                                    CTAs with a 2- or 3-stage TMA ring (tiles 64 x 16R, see
                                    PROBE_OPT_PIPE_ROWS), for the forward and the adjoint.  Every
                                    variant gives the same bits.  3D: 0 = one-barrier-per-plane
                                    kernels; 2 = pipelined kernels whose ring is refilled by a
                                    producer warp; 3 = pipelined kernels whose ring slot is refilled
                                    by the last compute warp done with it (no producer warp); by
                                    default the 3D autotuner picks 2 or 3, for the forward and the
                                    adjoint.  Setting it turns that choice off. */
    PROBE_OPT_DTT_HISTORY = 8,   /* 2D: 1 = keep Dtt u^n of every step in device memory instead of
                                    checkpointing and recomputing (FP32, W (nt-1) planes); 0 (default) */
    PROBE_OPT_AUTOTUNE = 9,      /* 1 (default): on the first call for a shape, time the 2D kernel variants
                                    (forward and adjoint kernel, pipeline depth, rows per thread, shot group)
                                    and keep the fastest; setting PROBE_OPT_PIPELINE, PROBE_OPT_PIPE_ROWS or
                                    PROBE_OPT_SHOT_GROUP turns it off */
    PROBE_OPT_PIPE_ROWS = 10,    /* 2D pipelined kernels: rows per thread R, tile 64 x 16R (1 or 2),
                                    forward and adjoint */
    PROBE_OPT_PIPELINE_ADJ = 11, /* adjoint kernel only (0, 2 or 3; PROBE_OPT_PIPELINE sets both).  3D: nonzero
                                    (default) = producer-warp adjoint with the receiver injection
                                    prebuilt per checkpoint segment, used when Kahan compensation
                                    is per segment or off; takes effect for workspaces sized after
                                    it is set */
    PROBE_OPT_PIPE_ROWS_ADJ = 12, /* 2D pipelined adjoint only: rows per thread (1 or 2) */
    PROBE_OPT_TBLOCK = 14,       /* 2D Born forward and checkpoint recompute: time levels advanced per
                                    launch, 1 or 2 (two levels: each CTA stages its tile with an 8-cell
                                    halo and recomputes the first level on the tile plus 4 cells, which
                                    halves the state traffic per level); 0 (default) = chosen by the
                                    autotuner.  Both give the same bits. */
    PROBE_OPT_OVERLAP3D = 16,    /* 3D Born forward: 1 (default) = the incident step n+1 runs on a second
                                    stream concurrently with the Born step n (the Dtt plane of the
                                    incident step is double-buffered), so each launch's last, partly
                                    filled wave of CTAs overlaps the other's; 0 = one stream.  Same
                                    bits either way. */
    PROBE_OPT_PLANES3D = 15,     /* 3D: z planes one CTA marches through (32, 64 or 128; each CTA loads
                                    8 halo planes besides them); 0 (default) = chosen by the autotuner,
                                    which times the forward step kernels on the real workspace at each
                                    value on the first call for a workload.  All values give the same
                                    bits. */
    PROBE_OPT_CLUSTER3D = 13     /* 3D thread-block-cluster kernels, a bit mask (default 0):
                                    bit 0 (1): the incident and Born fields of a column tile advance in
                                    one launch on a cluster of 1 + nb CTAs (nb <= 7), exchanging Dtt u0
                                    through distributed shared memory instead of HBM;
                                    bit 1 (2): the adjoint runs on clusters of PROBE_OPT_SHOT_GROUP shots
                                    (1, 2, 4 or 8; 0 = 4) whose imaging terms are summed in shared
                                    memory before one Kahan update of the group's image;
                                    0 = one field per CTA and separate incident and Born launches (the
                                    default: three CTAs per SM instead of two, measured faster) */
} probe_option;

/* Counters and timings of the last apply call (probe_get_stats). */
typedef struct {
    double ms_forward;           /* forward (incident + Born) sweeps, CUDA events */
    double ms_recompute;         /* checkpoint recompute sweeps */
    double ms_adjoint;           /* adjoint + imaging sweeps */
    double ms_total;             /* whole call on the device */
    long long launches_forward;  /* kernel launches in each sweep kind */
    long long launches_recompute;
    long long launches_adjoint;
    long long launches_total;    /* every kernel launch of the call */
    double cell_updates_forward; /* executed stencil cell-updates on the padded grid */
    double cell_updates_recompute;
    double cell_updates_adjoint;
    double bytes_forward;        /* algorithmic HBM bytes of each sweep kind */
    double bytes_recompute;
    double bytes_adjoint;
    int shot_wave;               /* shots resident per wave */
    int shot_group;              /* shots per CTA in the adjoint */
    int tile_z;                  /* 2D tile height used */
    int ckpt_stride;             /* checkpoint spacing used */
    int pipeline_forward;        /* 2D forward kernel: 0 one tile per CTA, 2..4 pipeline stages;
                                    3D: 0 one barrier per plane, 2 producer-warp refill, 3 refill by
                                    the last compute warp */
    int pipeline_adjoint;        /* 2D adjoint kernel: same encoding; 3D: as the forward, for the
                                    adjoint with the receiver injection from a per-segment band
                                    buffer */
    int dtt_history;             /* 1 when Dtt u^n of every step was kept instead of recomputed */
    int pipeline_rows;           /* rows per thread of the pipelined forward kernels (0: not pipelined) */
    int pipeline_rows_adjoint;   /* rows per thread of the pipelined adjoint kernel */
    int time_block;              /* 2D Born forward and recompute: time levels per launch (1 or 2) */
    int planes_3d;               /* 3D: z planes marched by one CTA (0 for 2D) */
    int pipeline_incident;       /* 3D: as pipeline_forward, for the incident step (forward and
                                    recompute; pipeline_forward then names the Born step's) */
} probe_stats;

/* Create a handle for one background model and acquisition geometry.
 * m0 [n...] interior slowness squared 1/c^2 (> 0, finite); src_idx [ns][ndim],
 * rec_idx [nr][ndim] interior node indices (several receivers may share a node);
 * wavelet [nt] source signature w(n dt) (Sec. 2: f_s = delta(x-s) w(t)).
 * Fails with PROBE_ERR_ARG on out-of-range indices, non-positive sizes or
 * spacing, or c_max dt / h_min above the stability limit of the scheme
 * (0.5547 in 2D, 0.4529 in 3D).  On success *out owns device memory until
 * probe_destroy. */
probe_status probe_create(probe_t* out, const probe_grid* grid, const float* m0,
                          int ns, const int* src_idx, int nr, const int* rec_idx,
                          const float* wavelet, int nt, double dt);

/* d = F dm: Born data of nb model perturbations (Sec. 2 linearised wave
 * equation).  dm [nb][n...] (interior), d [nb][ns][nt][nr]. */
probe_status probe_apply_F(probe_t h, const float* dm, float* d, int nb,
                           probe_stream_t stream);

/* img = F* d: exact adjoint of probe_apply_F (reverse-time migration, zero-lag
 * imaging condition, Sec. 1.1).  d [nb][ns][nt][nr], img [nb][n...]. */
probe_status probe_apply_Fadj(probe_t h, const float* d, float* img, int nb,
                              probe_stream_t stream);

/* Hdm = F*F dm summed over all shots (Sec. 1.1, H = F*F; Sec. 2 stack over
 * sources) for a batch of nb trial functions.  dm, Hdm [nb][n...]; may alias. */
probe_status probe_apply_H(probe_t h, const float* dm, float* Hdm, int nb,
                           probe_stream_t stream);

/* probe_apply_H on several models (of possibly different grid sizes) at once:
 * the sweeps of all models advance in the same kernel launches.  All models
 * must share nt, dt and the checkpoint stride.  dm[k], Hdm[k] are the arrays
 * of model k with nb[k] trials each.  nmodels <= 4. */
probe_status probe_apply_H_group(const probe_t* models, int nmodels,
                                 const float* const* dm, float* const* Hdm,
                                 const int* nb, probe_stream_t stream);

/* Randomized fit of Sec. 1.4: given trial functions y_j and x_j = H y_j
 * (j = 1..p, each [n...]), find the coefficients c (FP64, [P] with
 * P = nspatial * nangular * nradial <= 1024) minimising
 *     sum_j || y_j - sum_i c_i B_i x_j ||^2
 * (the least-squares problem whose normal equations M c = (Bx)^T y,
 * M_ik = sum_j (B_i x_j)^T (B_k x_j), Sec. 1.4 writes).  Solved on the device
 * in FP64 through a QR factorisation of the stacked columns A = [B_i x_j]
 * (CholeskyQR2: Cholesky QR with one reorthogonalisation), so the error grows
 * like cond(A) eps, not cond(A)^2 eps.  coeffs (host or device) and resid_rel
 * (||y - Bx c|| / ||y||, host) are written; the call synchronises.
 * Returns PROBE_ERR_STATE if the columns are numerically rank deficient. */
probe_status probe_fit(probe_t h, const probe_basis* basis, const float* y,
                       const float* Hy, int p, double* coeffs, double* resid_rel,
                       probe_stream_t stream);

/* out = sum_i c_i B_i img (end of Sec. 1.5).  coeffs [P] FP64, img and out
 * [n...]; img and out may alias. */
probe_status probe_apply_precond(probe_t h, const probe_basis* basis,
                                 const double* coeffs, const float* img, float* out,
                                 probe_stream_t stream);

/* Iterative solution of the linearised least-squares problem
 * min 1/2 ||F dm - d||^2 through its normal equations H dm = F*d (Sec. 2: the
 * fitted preconditioners are judged against gradient-descent iterations on
 * this functional, and preconditioned iterations apply the approximate inverse
 * to the migrated residual F*(d - F dm_k)).  rhs [n...] is the migrated image
 * F*d; x [n...] holds the start on entry (zeros allowed) and the last iterate
 * on return.  method PROBE_SOLVE_GD: steepest descent with exact line search,
 * step p.r / p.Hp along p = r_k, or along p = sum_i c_i B_i r_k when basis and
 * coeffs [P] (host, FP64) are given; PROBE_SOLVE_CG: conjugate gradients
 * (basis must be NULL).  r_k = rhs - H x_k is updated by the recurrence; its
 * 2-norms for k = 0..done go to resid [iters + 1] (host, FP64, may be NULL) and
 * the number of iterations performed to *done (may be NULL): fewer than iters
 * when the residual or the curvature p.Hp reaches zero.  Each iteration is one
 * probe_apply_H of one trial (plus one probe_apply_precond); inner products
 * are FP64 sums of FP32 products, read back every iteration, so the call
 * synchronises `stream`.  rhs and x may be host or device arrays. */
typedef enum { PROBE_SOLVE_GD = 0, PROBE_SOLVE_CG = 1 } probe_solve_method;
probe_status probe_solve(probe_t h, int method, int iters, const probe_basis* basis,
                         const double* coeffs, const float* rhs, float* x, double* resid,
                         int* done, probe_stream_t stream);

/* Krylov trial functions of the Kn preconditioners (Sec. 2, the comparison of
 * Krylov and randomized trial functions): y_1 = rhs / ||rhs|| (rhs normally the
 * migrated data F*d), x_j = H y_j, y_{j+1} = x_j / ||x_j|| for j = 1..n.
 * rhs [n_model]; y, Hy [n][n_model] receive the trials and their H
 * applications, ready for probe_fit (pairs (y_j, x_j)).  Each step is one
 * probe_apply_H of one trial; the norms are FP64 sums formed on the device.
 * Arrays may be host or device memory; the call synchronises `stream`. */
probe_status probe_krylov_trials(probe_t h, const float* rhs, int n, float* y, float* Hy,
                                 probe_stream_t stream);

/* Nonlinear prediction d = calF[m] (Sec. 1.1): the receiver traces of
 * m u_tt - Lap u = f_s for every shot; m [n...] interior (the sponge keeps the
 * values of m0), d [ns][nt][nr]. */
probe_status probe_forward_nonlinear(probe_t h, const float* m, float* d,
                                     probe_stream_t stream);

/* g = F*[m] resid: migration of the residual with the Born operator
 * linearised at m (Sec. 1.1: dJ/dm = -F*(d - calF[m]) = F*[m] (calF[m] - d)).
 * m, g [n...], resid [ns][nt][nr]. */
probe_status probe_gradient(probe_t h, const float* m, const float* resid, float* g,
                            probe_stream_t stream);

/* probe_apply_F without allocating: the same Born data as probe_apply_F, for
 * callers that must not allocate device memory during the call (a service that
 * has handed its remaining memory to its own pool, a framework that forbids
 * cudaMalloc/cudaFree between its own allocation points because they
 * synchronise the device, a real-time loop).  This operation has no
 * counterpart in the paper; it is an engineering variant of probe_apply_F.
 * Create the handle once beforehand (probe_create allocates its model arrays).
 * 2D handles only (a 3D handle gives PROBE_ERR_ARG).
 * dm [nb][n...] and d [nb][ns][nt][nr] must be device arrays.  The per-call
 * scratch is a library-internal static device array of 32 MiB, held on every
 * GPU that loads the library until the process exits; shots are processed in
 * waves that fit in it, and a call whose single shot does not fit
 * ((2 + 3 nb) padded planes of 4-byte cells) fails with PROBE_ERR_ARG.  The first
 * call on a device looks up the array's device address; make that call before
 * any stream capture.  All calls share the array: calls whose work overlaps on
 * the GPU race and must be serialised by the caller.  No cudaMalloc, cudaFree or
 * allocating library routine is called. */
probe_status probe_apply_F_noalloc(probe_t h, const float* dm, float* d, int nb,
                                   probe_stream_t stream);

/* Failure-detection check (no counterpart in the paper): launches one CTA
 * whose bounded mbarrier wait can never be satisfied, so it gives up after
 * timeout_ms (1..10000) of device time, records the timeout in the handle's
 * device error word and exits.  Returns PROBE_ERR_TIMEOUT (after synchronising
 * `stream`); the handle and the CUDA context remain usable.  This is the same
 * bounded-wait path every stencil kernel uses around its TMA loads. */
probe_status probe_diag_wait_timeout(probe_t h, int timeout_ms, probe_stream_t stream);

/* Set a tunable (probe_option); returns PROBE_ERR_ARG for unknown keys or values. */
probe_status probe_set_option(probe_t h, int key, long long value);

/* Copy the statistics of the last apply call (requires that call's stream to
 * have completed when timings are enabled). */
probe_status probe_get_stats(probe_t h, probe_stats* out);

/* Number of interior cells (prod n) and the padded-grid size, for callers
 * that size their own buffers. */
probe_status probe_sizes(probe_t h, long long* n_model, long long* n_padded, int* ns,
                         int* nr, int* nt);

/* Last error message of the handle (or of the last failed probe_create when
 * h is NULL).  Valid until the next call on the same handle. */
const char* probe_last_error(probe_t h);

/* Release every resource of the handle (safe on NULL). */
void probe_destroy(probe_t h);

/* Library version string. */
const char* probe_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PROBE_H */
