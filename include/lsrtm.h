/*
 * lsrtm.h — C ABI of the GB300 (sm_103a) multiparameter LSRTM operator library.
 *
 * The library applies the linearised Born modelling operator L and its exact
 * transpose L^T for the first-order velocity-pressure acoustic system
 * (Eq. 1: rho dv/dt + grad p = 0, kappa div v + dp/dt = f_p, kappa = rho Vp^2)
 * on a staggered grid, parametrised by m = (dln Vp, dln Ip) through
 * dln rho = dln Ip - dln Vp and dln kappa = dln Ip + dln Vp (Sec. 2), and
 * drives them with CGNR (Sec. 3) and PSF probes (App. D).
 *
 * Conventions shared by every entry point
 *   - Interior grid nz x (ny x) nx, x fastest; ny = 1 in 2D. A flat interior
 *     index is (iz*ny + iy)*nx + ix.
 *   - Models, perturbations and images are float32 arrays [nz][ny][nx]; a
 *     two-parameter array is [2][nz][ny][nx] with plane 0 = dln Vp and plane 1
 *     = dln Ip.
 *   - Data are float32 [nrec_total][nt], receiver-major, contiguous in time;
 *     receivers of shot s are rows rec_ptr[s] .. rec_ptr[s+1]-1. Sample n of a
 *     receiver is the pressure after time step n (time (n+1)*dt).
 *   - Array arguments may be device pointers or host pointers (pageable or
 *     pinned); the library detects host memory and stages it through its own
 *     device buffers. Geometry arrays are host pointers. The caller owns all
 *     arrays it passes; the library copies what it keeps.
 *   - All device work is queued on the handle's stream; calls return once the
 *     work is queued, except where a host result is returned (host output
 *     pointers, misfit history), in which case the call synchronises the stream.
 *   - Errors: every entry point returns an lsrtm_status; no exception crosses
 *     the ABI. lsrtm_last_error() gives a thread-local description of the last
 *     failure. Outputs are unspecified after an error.
 *   - Outputs are overwritten, never accumulated into.
 */
#ifndef LSRTM_H
#define LSRTM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LSRTM_OK = 0,
    LSRTM_ERR_ARG = 1,        /* invalid argument or configuration */
    LSRTM_ERR_CFL = 2,        /* time step violates the stability limit */
    LSRTM_ERR_GEOMETRY = 3,   /* source/receiver outside the interior grid */
    LSRTM_ERR_OOM = 4,        /* workspace exceeds the HBM budget or cudaMalloc failed */
    LSRTM_ERR_NONFINITE = 5,  /* NaN/Inf in an input or produced by a solve */
    LSRTM_ERR_CUDA = 6,       /* a CUDA runtime call failed (message in last_error) */
    LSRTM_ERR_STATE = 7       /* handle not usable for this call */
} lsrtm_status;

/* Storage precision of the saved boundary bands (App. A). The 16-bit formats
 * keep one FP32 scale per band per step: values are stored as v / s with s
 * the power of two that puts max|band| / s in [2^14, 2^15) (s >= 2^-126), so
 * the scaling is exact, FP16 keeps its 11-bit mantissa down to about 2^-23 of
 * each band's maximum and BF16 its 8-bit mantissa over the FP32 range. The
 * plain plan always stores FP32. */
enum { LSRTM_BAND_FP32 = 0, LSRTM_BAND_BF16 = 1, LSRTM_BAND_FP16 = 2 };
/* Source-wavefield reconstruction for L^T (App. A: the background field must
 * be available in reverse time). */
enum { LSRTM_RECON_BOUNDARY = 0,   /* boundary bands + reverse-time recomputation */
       LSRTM_RECON_CHECKPOINT = 1, /* full-state checkpoints + forward recomputation */
       LSRTM_RECON_AUTO = 2 };     /* boundary if it fits the budget, else checkpoints */
/* Execution plan. */
enum { LSRTM_PLAN_BATCHED = 0,     /* all shots of a batch per launch, CUDA graphs,
                                      background bands cached across calls */
       LSRTM_PLAN_PLAIN = 1 };     /* one shot per launch, no graph, background
                                      recomputed inside every L^T (reference plan) */

typedef struct {
    int ndim;                /* 2 or 3 */
    int nz, ny, nx;          /* interior grid (ny ignored in 2D) */
    double dz, dy, dx;       /* grid spacing [m] */
    double dt;               /* time step [s] */
    int nt;                  /* number of time steps */
    int fd_order;            /* 4 or 8: staggered Taylor order 2M */
    int npml;                /* CPML thickness in cells (>= fd_order/2) on every side */
    double f0;               /* dominant frequency [Hz]; sets the CPML alpha profile */
    double pml_vmax;         /* velocity for the CPML damping; <= 0: max of vp */
    int band_precision;      /* LSRTM_BAND_FP32, LSRTM_BAND_BF16 or LSRTM_BAND_FP16 */
    size_t hbm_budget_bytes; /* workspace cap; 0 = no cap */
    int recon_mode;          /* LSRTM_RECON_* */
    int plan;                /* LSRTM_PLAN_* */
    int shots_per_batch;     /* 0 = automatic */
    int wavelet_per_shot;    /* 0: wavelet [nt] shared; 1: wavelet [nshot][nt] */
    int checkpoint_interval; /* steps K between checkpoints in checkpoint mode;
                                0 = automatic (minimises checkpoint + segment-band memory) */
    int free_surface;        /* 1: free surface (p = 0) on the first interior row z = 0,
                                by the method of images: above it the pad holds the odd
                                mirror of p, the even mirror of v_z and the mirror of the
                                model, and has no CPML (a reading for the surface
                                acquisitions of Sec. 4-5); sources may not sit on that row,
                                receivers there record zero. 0: CPML on every side. */
    int guard_interval;      /* time steps between the non-finite guard's checks of the
                                wavefields: every that many steps of every time loop one
                                kernel scans the pressure planes of all slots of the batch
                                for NaN/Inf; on a hit it sets a device word, the remaining
                                time-step kernels of the loop return at once, and the call
                                (or the next call that synchronises) fails with
                                LSRTM_ERR_NONFINITE naming the loop and the step. CGNR
                                also checks its FP64 scalars every iteration and polls the
                                word one iteration behind. 0 = 64; < 0 = no wavefield checks. */
    int checkpoint_precision; /* storage of the checkpointed background states (checkpoint
                                reconstruction): LSRTM_BAND_FP32 (default; the images then equal
                                the boundary mode's bit for bit), LSRTM_BAND_BF16 or
                                LSRTM_BAND_FP16 with one FP32 scale per state plane per shot per
                                snapshot (the bands' power-of-two scaling), which halves the
                                checkpoint memory; the plain plan always stores FP32. */
} lsrtm_config;

typedef struct {
    int nshot;
    const int *src_idx;  /* host [nshot]: flat interior index of each shot's source */
    const int *rec_ptr;  /* host [nshot+1]: CSR offsets into rec_idx */
    const int *rec_idx;  /* host [rec_ptr[nshot]]: flat interior receiver indices */
    /* Optional per-shot aperture windows (2D, boundary-band reconstruction;
     * both NULL = every shot spans the model). Shot s is modelled on the
     * sub-model of interior columns [win_x0[s], win_x0[s] + win_nx[s]) with
     * its own CPML and edge replication of that sub-model; its source and
     * receivers must lie inside it, its records are that sub-problem's and
     * its image is added into those columns. The CPML damping uses the
     * configuration's pml_vmax for every shot. Shots of different window
     * widths advance in the same launches. */
    const int *win_x0;   /* host [nshot] first interior column, or NULL */
    const int *win_nx;   /* host [nshot] window width in columns, or NULL */
} lsrtm_geometry;

typedef struct lsrtm_handle lsrtm_handle;

/* Creates an operator handle: validates the configuration (CFL limit
 * dt <= 1 / (vmax sqrt(sum 1/h^2) sum|c_l|), geometry inside the interior),
 * pads the model by edge replication, derives kappa = rho vp^2 and the
 * staggered buoyancy (Eq. 1, Sec. 2), builds the CPML profiles and allocates
 * the workspace within hbm_budget_bytes.
 *   vp, rho : [nz][ny][nx] background velocity [m/s] and density [kg/m^3]
 *   wavelet : [nt] (or [nshot][nt]) source samples w(n dt); step n adds
 *             dt*w[n]/cell_volume to the pressure at the source node
 *   stream  : cudaStream_t to run on (NULL = legacy default stream)
 * The handle keeps copies; the caller may free its arrays afterwards. */
lsrtm_status lsrtm_create(const lsrtm_config *cfg, const float *vp, const float *rho,
                          const float *wavelet, const lsrtm_geometry *geom, void *stream,
                          lsrtm_handle **out);

/* Born modelling d = L dm (Eq. scattereqln with d = R dp, Sec. 3):
 *   dm : [2][nz][ny][nx] (dln Vp, dln Ip), supported on the interior
 *   d  : [nrec_total][nt] output */
lsrtm_status lsrtm_born(lsrtm_handle *h, const float *dm, float *d);

/* Migration g = L^T d: the exact transpose of lsrtm_born under the plain
 * Euclidean inner products, i.e. the zero-lag cross-correlations of
 * Eqs. (gradrho), (gradkappa) stacked over shots, mapped by the chain rule of
 * Sec. 3 (g_Vp = g_kappa - g_rho, g_Ip = g_kappa + g_rho).
 *   d           : [nrec_total][nt] input
 *   g           : [2][nz][ny][nx] output
 *   pseudo_hess : optional [nz][ny][nx] output of the pseudo-Hessian diagonal
 *                 of App. B (shared by both parameters), or NULL */
lsrtm_status lsrtm_adjoint(lsrtm_handle *h, const float *d, float *g, float *pseudo_hess);

/* Point-spread-function probe of App. D: psf = L^T L comb, where comb holds
 * unit spikes in plane `param` (0 = dln Vp, 1 = dln Ip) at every interior node
 * whose coordinates are all spacing/2 + k*spacing.
 *   psf : [2][nz][ny][nx] output */
lsrtm_status lsrtm_psf(lsrtm_handle *h, int param, int spacing, float *psf);

/* Remigration of App. E: out = L^T L m (m, out: [2][nz][ny][nx]). */
lsrtm_status lsrtm_remigrate(lsrtm_handle *h, const float *m, float *out);

/* Data-domain LSRTM (Sec. 3): CGNR on min ||L dm - d||^2, x0 = dm on entry,
 * restricted to the planes in param_mask (1 = dln Vp, 2 = dln Ip, 3 = both).
 * precond != 0 uses the diagonal pseudo-Hessian M = H + 1e-3 max(H) of App. B
 * (computed once). Krylov scalars and inner products are FP64 on the device.
 *   d      : [nrec_total][nt] observed data
 *   dm     : [2][nz][ny][nx] in: starting model, out: solution after niter
 *   misfit : host [niter+1] or NULL: ||d - L dm_k|| / ||d|| per iteration
 * Errors: LSRTM_ERR_NONFINITE when the guard (lsrtm_config.guard_interval)
 * finds NaN/Inf in a wavefield or a Krylov scalar, e.g. from NaN in d: the
 * solve stops at most one iteration after the hit, dm is not written. */
lsrtm_status lsrtm_cg_solve(lsrtm_handle *h, const float *d, float *dm, int niter, int precond,
                            int param_mask, double *misfit);

/* Step-wise CGNR with the same algorithm as lsrtm_cg_solve:
 * lsrtm_cg_begin computes r0 = d - L x0 and s0 = L^T r0 (x0 = NULL means 0),
 * lsrtm_cg_iterate performs niter iterations (each one L, one L^T and the
 * FP64 Krylov updates) and, if misfit is not NULL, synchronises and writes
 * the normalised misfit after each of them (host [niter]);
 * lsrtm_cg_result copies the current iterate to dm ([2][nz][ny][nx]) and,
 * if misfit0 is not NULL, the misfit of x0. Only one solve per handle is
 * active; lsrtm_cg_begin restarts it. lsrtm_cg_iterate returns
 * LSRTM_ERR_NONFINITE one iteration after the guard trips (the iteration
 * count then includes that iteration, whose time loops were skipped);
 * without a misfit buffer a hit in its last iteration is reported by the
 * next synchronising call (lsrtm_cg_result, lsrtm_synchronize). */
lsrtm_status lsrtm_cg_begin(lsrtm_handle *h, const float *d, const float *x0, int precond,
                            int param_mask);
lsrtm_status lsrtm_cg_iterate(lsrtm_handle *h, int niter, double *misfit);
lsrtm_status lsrtm_cg_result(lsrtm_handle *h, float *dm, double *misfit0);

/* Save and resume of a step-wise CGNR solve. lsrtm_cg_get_state copies the
 * state the next iteration reads: the iterate x and the search direction p
 * ([2][nz][ny][nx]), the data residual r ([nrec_total][nt]), the FP64
 * scalars {gamma = <s, M^-1 s>, <d, d>} and the iteration count (host or
 * device buffers; synchronous). To resume, call lsrtm_cg_begin with the same
 * d, precond and param_mask (it rebuilds the preconditioner and the misfit
 * normalisation), then lsrtm_cg_set_state with the saved state: the
 * following lsrtm_cg_iterate calls repeat the uninterrupted solve bit for
 * bit (the kernels are deterministic). Errors: LSRTM_ERR_STATE without an
 * active solve; LSRTM_ERR_ARG for a negative iteration count. */
lsrtm_status lsrtm_cg_get_state(lsrtm_handle *h, float *x, float *p, float *r, double *scalars, int *iter);
lsrtm_status lsrtm_cg_set_state(lsrtm_handle *h, const float *x, const float *p, const float *r,
                                const double *scalars, int iter);

/* Device-time accounting of the time loops, measured with CUDA events on the
 * library's own stream around each loop: born = fused background + Born
 * forward loops, background = background-only loops (band saving), adjoint =
 * reverse-time migration loops. launches = kernel launches those loops
 * contain (one per time step per batch); cells = padded cells advanced. */
typedef struct {
    double born_ms, background_ms, adjoint_ms;
    long long born_launches, background_launches, adjoint_launches;
    double born_cells, background_cells, adjoint_cells;
} lsrtm_timings;

/* Enables (1) or disables (0) the event timing of lsrtm_timings. */
lsrtm_status lsrtm_timing_enable(lsrtm_handle *h, int enable);

/* Synchronises the handle's stream and returns the accumulated timings;
 * reset != 0 clears them afterwards. */
lsrtm_status lsrtm_timing_read(lsrtm_handle *h, lsrtm_timings *out, int reset);

/* Born modelling without any device allocation, for callers that cannot
 * call cudaMalloc (host applications that own the GPU memory pool and forbid
 * foreign allocations, real-time loops where an allocation and the device
 * synchronisation it may cause are not allowed). The paper has no counterpart: this
 * is a deployment variant of lsrtm_born. It computes the same d = L dm for a
 * 2D grid, taking every byte of device workspace from one fixed 32 MiB
 * array that lives in this library's device image (each GPU that loads the
 * library holds it until exit), and calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *   cfg     : as for lsrtm_create; 2D only, and cfg->pml_vmax must be > 0
 *   vp, rho, wavelet, dm : device pointers (layouts as for lsrtm_create / lsrtm_born)
 *   geom    : host arrays, as for lsrtm_create; copied with cudaMemcpyAsync
 *             before the call returns, so they may be freed afterwards
 *   d       : device pointer, [nrec_total][nt] output
 *   stream  : cudaStream_t for all the work (NULL = legacy default stream)
 * Problems whose workspace exceeds 32 MiB are rejected with LSRTM_ERR_OOM
 * and a message giving the size needed. All calls on a device share the
 * array and leave their contents in it; each call re-initialises what it
 * reads, but calls whose GPU work overlaps race, so order them. The first
 * call on a device looks up the array's device address and configures the
 * kernels; make it before any stream capture. Inputs are not checked for
 * finiteness (a non-finite model gives non-finite records, not an error).
 * Returns once the work is queued. */
lsrtm_status lsrtm_born_static(const lsrtm_config *cfg, const float *vp, const float *rho,
                               const float *wavelet, const lsrtm_geometry *geom, const float *dm,
                               float *d, void *stream);

/* Nonlinear modelling (Eq. 1) in the handle's own model (vp, rho given at
 * creation; aperture windows as for lsrtm_born): d[r][n] = p^{n+1} at the
 * receiver node, the same recording as lsrtm_born with the pressure in place
 * of its perturbation. Observed data come from a handle created on the true
 * model, synthetic background data from one on the background model.
 *   d : [nrec_total][nt] output (host or device)
 * Asynchronous for device outputs. */
lsrtm_status lsrtm_model(lsrtm_handle *h, float *d);

/* Muted data residual, the data-domain input of Sec. 4: observed minus
 * background data times a mask that removes the direct arrivals and the
 * long-offset refractions. Per receiver r (horizontal source-receiver offset
 * o_r = |(x_r - x_s, y_r - y_s)| in metres) and sample n (t_n = (n + 1) dt):
 *     d_out = ramp(t_n - o_r / v_mute - t0, t_taper) ramp(o_max - o_r, o_taper)
 *             (d_obs - d_syn),
 *     ramp(u, W) = 0 for u <= 0, 1 for u >= W, (1 - cos(pi u / W)) / 2 between
 *     (W = 0: a step); no far-offset cut when o_max <= 0.
 * The mute times are formed in FP64; the data arithmetic is FP32.
 *   d_obs, d_syn : [nrec_total][nt] (host or device; d_syn may be NULL)
 *   v_mute (m/s) > 0, t0 (s), t_taper (s) >= 0, o_max (m), o_taper (m) >= 0
 *   d_out        : [nrec_total][nt] output (host or device; may be d_obs)
 * Errors: LSRTM_ERR_ARG for out-of-range parameters. Synchronous. */
lsrtm_status lsrtm_mute_residual(lsrtm_handle *h, const float *d_obs, const float *d_syn, double v_mute, double t0,
                                 double t_taper, double o_max, double o_taper, float *d_out);

/* Waits for all work queued by the handle and reports a failure that a
 * kernel recorded on the device: a bounded wait for its tile copies that
 * gave up, or a refused misaligned copy, as LSRTM_ERR_CUDA; a tripped
 * non-finite guard (lsrtm_config.guard_interval) as LSRTM_ERR_NONFINITE. The
 * record is cleared. Operator calls are asynchronous, so such a failure surfaces here
 * or at the next synchronous call. The paper has no counterpart: this is
 * host-side error handling. */
lsrtm_status lsrtm_synchronize(lsrtm_handle *h);

/* Replaces the stream used by later calls. */
lsrtm_status lsrtm_set_stream(lsrtm_handle *h, void *stream);

/* Nonstationary deblurring (image-domain LSRTM, App. E) of a 2D image pair.
 * App. E connects the reference image m' = m_rtm and the remigrated image
 * m'' = L^T L m' by a convolution with the inverse of a locally
 * translation-invariant Hessian. Per comb node (z_k, x_k) = (s/2 + i s,
 * s/2 + j s) a flen x flen filter f_k minimises, over the pixels p within s
 * of the node (clipped to the image),
 *     sum_p ((f * m'')(p) - m'(p))^2 + eps_k ||f||^2,
 *     (f * g)(p) = sum_{|a|,|b|<=flen/2} f[a][b] g(p - (a, b)), g = 0 outside,
 *     eps_k = eps * trace(A^T A) / flen^2,
 * through FP64 normal equations and a Cholesky factorisation (a window with
 * m'' = 0 gets the zero filter). Then
 *     dm_out = sum_k w_k (f_k * m_rtm) / sum_k w_k,
 *     w_k(p) = max(0, 1 - |z - z_k|/s) max(0, 1 - |x - x_k|/s),
 * each parameter plane filtered on its own (FP32 apply).
 *   m_rtm, m_remig : [2][nz][nx] (host or device; read only)
 *   spacing s      : node spacing and window half-width, 2 <= s <= 48
 *   flen           : odd filter length, 1 <= flen <= 11
 *   eps            : relative Tikhonov weight (>= 0; 1e-3 is typical)
 *   dm_out         : [2][nz][nx] output (host or device)
 *   filters        : optional [2][nkz][nkx][flen][flen] output, nk = number
 *                    of nodes along the axis (NULL to skip)
 * Errors: LSRTM_ERR_ARG for 3D handles or parameters out of range;
 * LSRTM_ERR_NONFINITE if a factorisation met a non-positive pivot (those
 * filters are zero; the other outputs are written). Synchronous. */
lsrtm_status lsrtm_deblur(lsrtm_handle *h, const float *m_rtm, const float *m_remig, int spacing, int flen,
                          double eps, float *dm_out, float *filters);

/* Nonstationary Wiener deblurring, the Fourier form of App. E. Within a local
 * block the Hessian is taken as circulant, H = F^H Lam F, and dm = F^H Lam^-1
 * F m_rtm (Eq. sol) with Lam^-1 from the regularised least squares of App. E,
 * the Wiener ratio Lam_i^-1 = conj([F m'']_i) [F m']_i / (|[F m'']_i|^2 + eps_k),
 * m' = m_rtm, m'' = L^T L m'. Blocks: per comb node (z_k, x_k) = (s/2 + i s,
 * s/2 + j s) the 2s x 2s pixels z_k - s .. z_k + s - 1 (same in x), zero
 * outside the image; F is the block's 2D DFT; eps_k = eps * mean_i |[F m'']_i|^2
 * (a block with m'' = 0 gives 0); block results are blended with the bilinear
 * valence w_k = max(0, 1 - |z - z_k|/s) max(0, 1 - |x - x_k|/s); each
 * parameter plane on its own. FP32 DFTs.
 *   m_rtm, m_remig : [2][nz][nx] (host or device; read only)
 *   spacing s      : 2 <= s <= 32
 *   eps            : relative stabiliser, > 0 (1e-3 is typical)
 *   dm_out         : [2][nz][nx] output (host or device)
 * Errors: LSRTM_ERR_ARG for 3D handles or parameters out of range.
 * Asynchronous for device outputs. */
lsrtm_status lsrtm_deblur_wiener(lsrtm_handle *h, const float *m_rtm, const float *m_remig, int spacing, double eps,
                                 float *dm_out);

/* Interpolated PSF Hessian (migration deconvolution with PSFs, App. D) of a
 * 2D or 3D image. The PSF image of a spike comb (nodes s/2 + k s along both axes,
 * as lsrtm_psf places them) holds a localised Hessian column around each
 * node; the column at any pixel c is interpolated from the windows of the
 * (up to) four surrounding nodes with the weights of Eq. (trilinear), 2D form:
 *     H(c + a, c) = sum_corners w_corner(c) Q(node_corner + a),
 *     |a_z|, |a_x| <= half,  Q = 0 outside the image,
 *     1D weights (1 - w, w), w = (c - node_k0) / s between the first and the
 *     last node; beyond them the nearest end node alone (w = 0),
 * entries with c + a outside the image dropped. In 3D the column takes the
 * eight corners of the node cell with the products of the three 1D weights
 * (Eq. trilinear as printed) and windows of (2 half + 1)^3 voxels; nz <= 65535.
 * Block (i, j) of the two-
 * parameter Hessian (output plane i, input plane j; 0 = Vp, 1 = Ip) takes Q
 * = plane i of the PSF of the comb in parameter j. The operator applied is
 * P H P, P keeping the planes of param_mask; it is formed on the fly (never
 * stored).
 *   psf_vp, psf_ip : [2][nz][ny][nx] PSF images of the combs in Vp and Ip (host
 *                    or device; read only). The one of a parameter outside
 *                    param_mask may be NULL.
 *   spacing s      : comb spacing, 2 <= s <= 64
 *   half           : window half-width, 0 <= half <= 15; < 0 selects
 *                    (s - 1) / 2 (the widest window clear of the neighbours')
 *   param_mask     : 1 Vp, 2 Ip, 3 both
 *   transpose      : 0 for y = P H P x, 1 for y = P H^T P x
 *   x, y           : [2][nz][ny][nx] (host or device, not overlapping); planes
 *                    outside param_mask are ignored in x and zero in y
 * Errors: LSRTM_ERR_ARG for parameters out of range, a missing PSF, an image
 * without comb nodes or overlapping x and y. Asynchronous for device outputs. */
lsrtm_status lsrtm_psf_hessian(lsrtm_handle *h, const float *psf_vp, const float *psf_ip, int spacing, int half,
                               int param_mask, int transpose, const float *x, float *y);

/* Image-domain least squares with the interpolated PSF Hessian (App. D):
 * CGNR (CGLS form, FP64 scalars) on H^H H dm = H^H P m_rtm from dm = 0, for
 * niter iterations; the interpolated H is singular in general, and from zero
 * CGNR tends to the minimum-norm least-squares solution.
 *   psf_vp, psf_ip, spacing, half, param_mask : as for lsrtm_psf_hessian
 *   m_rtm   : [2][nz][ny][nx] migrated image (host or device; read only)
 *   dm      : [2][nz][ny][nx] output (host or device)
 *   misfit  : optional host [niter + 1], ||P m_rtm - H dm_k|| / ||P m_rtm||
 * Errors: as lsrtm_psf_hessian; LSRTM_ERR_NONFINITE if the solution is not
 * finite. Synchronous. */
lsrtm_status lsrtm_psf_cg(lsrtm_handle *h, const float *psf_vp, const float *psf_ip, int spacing, int half,
                          int param_mask, const float *m_rtm, float *dm, int niter, double *misfit);

/* Bytes of device workspace the handle holds. */
size_t lsrtm_workspace_bytes(const lsrtm_handle *h);

/* Autotuner of the Born and migration time-step kernels (no counterpart in
 * the paper). A CTA of the 2D kernels owns a fixed number of x-columns, one
 * of the fused 3D kernels a fixed (x, y) tile, and marches down a chunk of
 * tzc padded rows; more chunks give more CTAs per shot but repeat 2M
 * warm-up rows per chunk. The tuner times `steps` Born and migration steps
 * (0: 16) on the first batch for every split of the padded depth into 1..12
 * chunks of at least 2M + 8 rows (and the current one), keeps the fastest
 * and rebuilds the receiver tiling; results do not depend on the choice
 * (every cell is computed the same way). Captured graphs and the cached
 * background are dropped. Outputs (each may be NULL):
 *   *tzc      chosen rows per chunk
 *   ms        [2*ncand] pairs (tzc, ms per Born + migration step); room for
 *             at least 2*13 doubles
 *   *ncand    number of candidates timed
 * Synchronous; it uses the handle's slots as scratch. */
lsrtm_status lsrtm_autotune(lsrtm_handle *h, int steps, int *tzc, double *ms, int *ncand);

/* How the handle reconstructs the background in reverse time (chosen at
 * creation from recon_mode and the memory available):
 *   *mode     LSRTM_RECON_BOUNDARY or LSRTM_RECON_CHECKPOINT (never AUTO)
 *   *interval checkpoint interval K (0 in boundary mode)
 *   *batch    shots per batch
 * Any output pointer may be NULL. Returns LSRTM_ERR_ARG for a NULL handle. */
lsrtm_status lsrtm_reconstruction(const lsrtm_handle *h, int *mode, int *interval, int *batch);

/* Kernel launches issued by this handle since creation (graph replays count
 * every kernel node they contain). */
long long lsrtm_kernel_launches(const lsrtm_handle *h);

/* Releases the handle and its workspace (NULL is ignored). */
void lsrtm_destroy(lsrtm_handle *h);

/* Thread-local description of the last error ("" if none). */
const char *lsrtm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LSRTM_H */
