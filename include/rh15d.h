/*
 * rh15d.h -- C ABI of librh15d_gpu.so: the column-by-column (1.5D) multi-level
 * accelerated Lambda iteration (MALI) on one NVIDIA GB300 (sm_103a).
 *
 * The problem (Pereira & Uitenbroek, RH 1.5D, Sect. 2): a model atom and many
 * atmosphere columns go in; every column is an independent plane-parallel NLTE
 * problem (Sect. 2.2) iterated to its own convergence (Sect. 2.3); converged
 * level populations and the vertical emergent spectrum (Sect. 2.2) come out.
 * The method (Sect. 2.1): MALI with a local (diagonal) approximate Psi
 * operator and preconditioned rate equations, overlapping transitions sharing
 * opacity and emissivity, Ng acceleration (Sect. 2.3), LTE start (Sect. 2.3).
 *
 * Conventions (all functions):
 *   - return an rh_status; no exception or abort crosses the ABI;
 *   - host pointers are read (inputs) or written (outputs) during the call
 *     only, the library keeps no reference to them; the library copies;
 *   - the context owns all device memory it allocates and frees it in
 *     rh_destroy;
 *   - calls on one context are not thread-safe; distinct contexts are
 *     independent;
 *   - all arrays are C-contiguous, SI units, depth index k = 0 at the TOP;
 *   - after an error, rh_last_error() returns a message naming the first bad
 *     argument (e.g. the first bad column and depth).
 * Nothing here needs PyTorch; the Python binding passes plain pointers.
 */
#ifndef RH15D_H
#define RH15D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rh_ctx rh_ctx;

typedef enum {
    RH_OK = 0,
    RH_EINVAL = 1,     /* invalid argument or input value */
    RH_ENOMEM = 2,     /* device or host allocation failed */
    RH_ECUDA = 3,      /* a CUDA runtime call or kernel failed */
    RH_ESTATE = 4,     /* call out of order (e.g. iterate before load) */
    RH_ETIMEOUT = 5,   /* a bounded device wait gave up */
    RH_ENOTCONV = 6    /* informational: some columns did not converge */
} rh_status;

/* per-column status codes written by rh_iterate */
enum { RH_COL_CONVERGED = 0, RH_COL_MAXITER = 1, RH_COL_NONFINITE = 2, RH_COL_SINGULAR = 3,
       RH_COL_NOTRUN = 4 };

/* Create a context on CUDA device `cuda_device`.  `cuda_stream` is a
 * cudaStream_t to launch on (NULL: the context creates its own stream).
 * The caller keeps ownership of a stream it passes. */
int rh_create(rh_ctx **out, int cuda_device, void *cuda_stream);
void rh_destroy(rh_ctx *ctx);
/* Message of the last failed call on this context (never NULL; valid until
 * the next call on the context). */
const char *rh_last_error(const rh_ctx *ctx);

/* ---------------------------------------------------------------------- */
/* Model atom (Sect. 2.1: multi-level atom with bound-bound and bound-free  */
/* transitions).  Levels are indexed from the ground level; the last level  */
/* is the continuum (ionised stage).  Every bound-free transition goes from  */
/* cont_l[q] to the last level.                                              */
typedef struct {
    int32_t nlev;                  /* levels including the continuum, 2..8 */
    const double *E_J;             /* [nlev] energy above the ground level, J */
    const double *g;               /* [nlev] statistical weights (> 0) */
    int32_t nline;                 /* bound-bound transitions */
    const int32_t *line_l, *line_u;/* [nline] lower < upper < nlev-1 */
    const double *line_f;          /* [nline] absorption oscillator strength */
    const double *line_a_top;      /* [nline] Voigt damping at k = 0 */
    const double *line_a_bot;      /* [nline] Voigt damping at k = ndep-1 (log-interpolated in k) */
    const int32_t *line_nlambda;   /* [nline] wavelength points of the line (>= 2) */
    const double *line_qwing;      /* [nline] half-width of the line grid, Doppler widths at T_ref */
    int32_t ncont;                 /* bound-free transitions */
    const int32_t *cont_l;         /* [ncont] lower level */
    const double *cont_alpha0;     /* [ncont] cross section at the edge, m^2 (Kramers nu^-3 law) */
    const int32_t *cont_nlambda;   /* [ncont] wavelength points (>= 2) */
    const double *cont_ratio;      /* [ncont] range: edge frequency .. ratio * edge (> 1) */
    double mass_amu;               /* atomic mass, amu */
    double T_ref;                  /* K, reference temperature of the line grids */
    int32_t nmu;                   /* Gauss-Legendre angles on (0,1], 1..8 */
    double metal_floor;            /* electrons per hydrogen atom from metals */
    const int32_t *line_prd;       /* [nline] 1: angle-averaged partial redistribution (Hummer R_II-A),
                                      NULL or 0: complete redistribution; at most 4 PRD lines, no two
                                      sharing a wavelength point */
} rh_atom_desc;

/* Copy the atom, build the wavelength grid (line bands on a sinh-stretched
 * symmetric grid, continua geometric in frequency), the per-wavelength lists
 * of overlapping transitions (Sect. 2.1), quadrature weights, and upload the
 * tables.  RH_ESTATE if columns are loaded.  RH_EINVAL for a descriptor out
 * of range (more than 3 transitions overlapping at one wavelength, more
 * than 32 transitions, nlev > 8, nmu > 8, Voigt damping above 0.05). */
int rh_setup_atom(rh_ctx *ctx, const rh_atom_desc *desc);

/* Number of wavelength points of the grid (0 before rh_setup_atom). */
int64_t rh_nlambda(const rh_ctx *ctx);
/* Copy the grid frequencies [nlambda] (Hz) into nu_out (host). */
int rh_get_grid(const rh_ctx *ctx, double *nu_out);

/* ---------------------------------------------------------------------- */
/* Load ncol columns of ndep depth points (Sect. 2.2: one column = one       */
/* independent 1D problem).  Layout [ncol][ndep], k = 0 at the top, z        */
/* strictly decreasing with k.  ne_m3 may be NULL: n_e then comes from       */
/* hydrogen Saha ionisation plus metal_floor * n_H electrons.  on_device = 0: */
/* host pointers, copied; on_device = 1: device pointers, copied on the       */
/* context's stream (the caller keeps ownership).  Computes the LTE           */
/* populations n*, collisional rates and the LTE start.  RH_EINVAL names the  */
/* first non-finite or non-positive T, n_H (n_e), or non-decreasing z.        */
int rh_load_columns(rh_ctx *ctx, int64_t ncol, int32_t ndep, const double *z_m,
                    const double *T_K, const double *ne_m3, const double *nH_m3,
                    const double *vz_ms, int32_t on_device);

/* ---------------------------------------------------------------------- */
typedef struct {
    int32_t maxiter;      /* formal solutions per column (default 500) */
    double tol;           /* stop when max_{i,k} |dn/n| < tol (Sect. 2.3: 1e-3) */
    int32_t ng_order;     /* 0 (off) or 2 (Ng 1974, Sect. 2.3) */
    int32_t ng_delay;     /* first acceleration at this iteration */
    int32_t ng_period;    /* iterations between accelerations */
    int32_t start;        /* 0: LTE populations; 1: learned initial guess (rh_surrogate_*),
                             LTE where its prediction is not finite; 2: populations set by
                             rh_set_populations or left by the previous rh_iterate;
                             3: zero radiation; 4: escape probability iterations
                             (Sect. 2.3; see rh_start_populations) */
    int32_t precision;    /* 0: all FP64; 1: FP32 formal solution and rates, FP64 solve and Ng */
    int32_t persistent;   /* 0: static split of columns over resident blocks (normal mode,
                             Sect. 3.1); 1: device work queue (pool mode, Sect. 3.1) */
    int32_t block_warps;  /* warps per block (0: library default) */
    double crsw_init;     /* collisional-radiative switching (Hummer & Voels 1988, Sect. 2.3):
                             collisional rates scaled by max(1, crsw_init 10^-(it-1)); <= 1: off */
    int32_t only_unconverged; /* 1: iterate only the columns whose status is not RH_COL_CONVERGED
                             (Sect. 2.3: re-run the columns that did not converge with other
                             options); converged columns are left untouched */
    double prd_eps0;      /* PRD switching (Eq. 1): rho' = eps rho + (1 - eps), eps = min(1, eps0 it^2);
                             <= 0: off (eps = 1).  Atoms with PRD lines only */
    int32_t prd_hybrid;   /* PRD lines: 0 angle-averaged redistribution in the static frame; 1 the
                             hybrid approximation of angle-dependent PRD in moving atmospheres
                             (Sect. 2.1): rho is computed in the frame of the moving gas from the
                             gas-frame mean intensity J_f(nu) = sum over rays (w_mu/2)
                             I(nu + nu0 mu_z v_z / c), and each ray emits with rho_f(nu - nu0
                             mu_z v_z / c); both transfers interpolate linearly in frequency over
                             the line's points, constant beyond its ends.  Without velocities the
                             two are the same scheme */
    int32_t formal;       /* formal solver of the iteration: 0 linear short characteristics (Olson &
                             Kunasz 1987); 1 quadratic Bezier short characteristics (the paper names no
                             scheme): between the upwind point u and the point o the source function
                             is the Bezier curve with control point C = S_o - (dtau_u/2) S'_o, S'_o the
                             Fritsch-Butland harmonic mean of the slopes to u and to the downwind
                             point (0 where they differ in sign), C held between S_u and S_o and the
                             midpoint without a downwind point; Psi* = w_o + w_c.  Exact for a
                             source function linear in tau, third order for smooth ones.  Emergent
                             spectra (rh_emergent_spectrum, rh_emergent_stokes) keep their own
                             solvers */
} rh_iter_opts;

typedef struct {
    int64_t n_converged, n_maxiter, n_failed;   /* over all loaded columns, after the call */
    int64_t n_processed;           /* columns iterated by this call */
    int64_t iterations_total;      /* sum over the processed columns of formal solutions */
    double seconds;                /* device time of the iteration kernel */
    double pts;                    /* depth x lambda x mu points solved */
    double max_dn_final;           /* max over columns of the last max |dn/n| (NaN entries skipped) */
    int64_t guess_fallback_depths; /* start = 1: depths whose prediction fell back to LTE */
    double guess_seconds;          /* start = 1: time of the prediction (included in seconds) */
} rh_iter_stats;

/* Iterate every loaded column to convergence or maxiter.  Writes per-column
 * populations, iteration counts, status and last max|dn/n| (read them with
 * rh_get_populations).  Returns RH_OK, or RH_ENOTCONV if any column did not
 * converge (results are still valid for the converged ones). */
int rh_iterate(rh_ctx *ctx, const rh_iter_opts *opts, rh_iter_stats *stats_out);

/* ---------------------------------------------------------------------- */
/* Emergent Stokes vector I, Q, U, V at mu = 1 (vertical ray, Sect. 2.2) of  */
/* line `line` (index among the lines of the atom) with Zeeman splitting of  */
/* a normal triplet of effective Lande factor g_eff, for the current         */
/* populations; the paper's 1.5D final spectra with a magnetic field         */
/* (Sect. 1, Stokes vector).  Field strength B_T [T], inclination theta to   */
/* the vertical and azimuth chi [rad] per depth, layout [ncol][ndep] (host,  */
/* or device when on_device = 1).  The line's propagation matrix and        */
/* emission follow Landi Degl'Innocenti & Landolfi (2004) without atomic     */
/* polarisation (source function S_l = n_u A/(n_l B_lu - n_u B_ul) for all   */
/* components); the background and other transitions are unpolarised.       */
/* Formal solver DELO-linear (Rees, Durrant & Murphy 1989); bottom boundary  */
/* I = B + dB/dtau, Q = U = V = 0.  With B_T = 0 the result equals           */
/* rh_emergent_spectrum at mu = 1 (I) and Q = U = V = 0.  iquv_out           */
/* [ncol][nlambda][4] (host, or device when on_device = 1).  precision 0:    */
/* FP64; 1: FP32 profiles and solver (opacities FP64).                       */
int rh_emergent_stokes(rh_ctx *ctx, int32_t line, double g_eff, const double *B_T, const double *theta,
                       const double *chi, int64_t nlambda, const double *lambda_m, double *iquv_out,
                       int32_t precision, int32_t on_device);

/* ---------------------------------------------------------------------- */
/* ---------------------------------------------------------------------- */
/* Depth-grid optimisation (Sect. 2.3: the atmosphere of each column is      */
/* interpolated onto a grid with more points where temperature, velocity or  */
/* optical depth change fastest, optionally without the upper layers).  The  */
/* paper gives no formula; this library's reading: every loaded column is    */
/* replaced by ndep_out points (2..4096) equidistant in the monitor s, whose */
/* step between neighbouring points is                                       */
/*   sqrt((d log10 N_H / dlog_colden)^2 + (d ln T / dlnT)^2                   */
/*        + (d v_z / dvz)^2 + (d z / dz_max)^2),                              */
/* N_H(z) the hydrogen column density above z (the optical-depth proxy; n_H   */
/* H at the top point, H the scale height of the top two points, plus the   */
/* exact integral of an exponential n_H between points), dz_max =           */
/* spacing_factor x column height / (ndep_out - 1).  The ends of the column  */
/* are kept; with use_z_top the layers above z_top (m) are removed first,    */
/* the new top point at z_top.  T and v_z are interpolated linearly, n_H and */
/* n_e logarithmically in height; then the columns are loaded as by          */
/* rh_load_columns (LTE populations, rates; populations reset).  Typical     */
/* scales: 0.1 dex, 0.02, 1000 m/s, 4.  RH_EINVAL for bad options or a      */
/* z_top at or below a column's bottom (naming the first such column).      */
typedef struct {
    double dlog_colden, dlnT, dvz, spacing_factor, z_top;
    int32_t use_z_top;
} rh_grid_opts;
int rh_regrid(rh_ctx *ctx, int32_t ndep_out, const rh_grid_opts *opts);
/* The loaded atmosphere [ncol][ndep] into host buffers (any may be NULL). */
int rh_get_columns(rh_ctx *ctx, double *z_out, double *T_out, double *nH_out, double *vz_out);

/* Start solutions (Sect. 2.3: "LTE populations, zero radiation, and ...     */
/* escape probability iterations"), written into the current populations of */
/* every loaded column (iterate from them with start = 2).  kind 0: LTE.     */
/* kind 1, the learned guess of start = 1 (no counterpart in the paper): the */
/* network's ln b per level and depth, n = e^{ln b} n* renormalised per      */
/* depth to sum n = n_H, LTE at a depth with a non-finite prediction;        */
/* RH_ESTATE without a network for the loaded depth count.                   */
/* kind 3, zero radiation: the rate equations with J = 0 -- radiative rates  */
/* are spontaneous only (A_ul; for a continuum the recombination            */
/* 4 pi sum w (2 h nu^3/c^2) alpha (n*_l/n*_c) e^{-h nu/kT} / (h nu) over its */
/* wavelength points) -- plus collisions, solved once per depth.  kind 4,    */
/* escape probability: from LTE, 3 solves of the same equations with each    */
/* spontaneous rate multiplied by the probability of escape through the top  */
/* p = beta(tau)/2, beta(tau) = (1 - e^{-tau})/tau, tau the line-centre       */
/* (Doppler core) or edge optical depth from the top at the previous         */
/* populations.  FP64.  Status of each column: RH_COL_NOTRUN, or             */
/* RH_COL_SINGULAR where a solve failed (its populations are then LTE).      */
int rh_start_populations(rh_ctx *ctx, int32_t kind);

/* ---------------------------------------------------------------------- */
/* The paper's two-stage strategy as one call (Sect. 2.3: aggressive       */
/* options first, then the columns that did not converge again with other  */
/* options).  Pass 1 iterates every column with `pass1` (start 0, 1 or 2;  */
/* only_unconverged is ignored).  Then, for r = 0 .. nrerun-1, the columns  */
/* whose status is not RH_COL_CONVERGED are iterated again from LTE with    */
/* collisional-radiative switching factor rerun_crsw[r] (>= 1; 1: none),     */
/* Ng as rerun_ng[r] says and rerun_maxiter iterations -- inside the column */
/* kernel (fused_rerun = 1)                                                  */
/* or as separate passes over a device-selected list.  No host round trip   */
/* happens between the passes.                                             */
/* use_graph = 1: the whole sequence (learned guess, pass 1, selections,    */
/* re-run passes, counters) is captured into a CUDA graph on the first call */
/* and the instantiated graph is replayed by later calls while the loaded   */
/* columns, the options, the lane table and the network are the same        */
/* objects; it is re-captured otherwise.  The context's stream must not be  */
/* the legacy default stream for capture (rh_create with NULL makes its own */
/* stream).  autotune = 1: before the first solve for this precision,       */
/* rh_autotune runs on the loaded columns (unless a tuning is present) and   */
/* its choice is used whenever pass1.block_warps is 0.                       */
/* Returns RH_OK, or RH_ENOTCONV if columns remain unconverged after all     */
/* passes (their results are those of the last pass that iterated them).    */
#define RH_MAX_RERUN 4
typedef struct {
    rh_iter_opts pass1;
    int32_t nrerun;                    /* 0 .. RH_MAX_RERUN */
    int32_t rerun_maxiter;             /* iterations of each re-run pass (>= 1) */
    double rerun_crsw[RH_MAX_RERUN];   /* switching factor of each re-run pass (>= 1; 1: none) */
    int32_t use_graph;                 /* 1: capture / replay a CUDA graph */
    int32_t autotune;                  /* 1: tune the launch shape once (see rh_autotune) */
    int32_t rerun_ng[RH_MAX_RERUN];    /* 1: Ng acceleration in that re-run pass (pass 1's order,
                                          delay and period); 0: none (the usual choice together
                                          with collisional-radiative switching) */
    int32_t fused_rerun;               /* 1: the column kernel runs the re-run ladder itself: a block
                                          whose column does not converge restarts it at once with the
                                          next re-run options, overlapping the rest of pass 1 (same
                                          per-column results as separate passes); 0: one kernel
                                          launch per pass, the selection done by a device kernel */
} rh_solve_opts;

typedef struct {
    int64_t n_converged, n_maxiter, n_failed;  /* after all passes */
    int64_t iterations_total;          /* formal solutions over all passes */
    int64_t pass_columns[1 + RH_MAX_RERUN];    /* columns entering each pass */
    int64_t pass_iterations[1 + RH_MAX_RERUN]; /* formal solutions of each pass */
    double seconds;                    /* device time of the whole sequence */
    double pass_seconds[1 + RH_MAX_RERUN]; /* device time of each pass (pass 1 includes the guess;
                                          with fused_rerun the re-runs are inside pass 1) */
    double pts;                        /* depth x lambda x mu points solved */
    int64_t guess_fallback_depths;     /* start = 1: depths that fell back to LTE */
    int32_t kernel_launches;           /* kernels launched by the sequence */
    int32_t graph_replayed;            /* 1: an instantiated graph was replayed */
    int32_t block_warps, ctas_per_sm;  /* launch shape used for the column kernel */
} rh_solve_stats;

int rh_solve(rh_ctx *ctx, const rh_solve_opts *opts, rh_solve_stats *stats_out);

/* Launch-shape autotuner for the column kernel (the ray tile is fixed at   */
/* 32 wavelengths x 1 angle per warp; what is tuned is the warps per column */
/* block and the column blocks resident per SM).  Times every candidate on  */
/* up to 4 x SMs of the loaded columns for 2 iterations from LTE in         */
/* `precision`, restores those columns' populations and results, and keeps  */
/* the fastest for that precision in the context (dropped by rh_setup_atom  */
/* and by rh_load_columns with another ndep).  cand_* receive up to          */
/* RH_MAX_TUNE candidates (ms = -1: did not fit).                            */
#define RH_MAX_TUNE 8
typedef struct {
    int32_t best_block_warps, best_ctas_per_sm;
    int32_t ncand;
    int32_t cand_block_warps[RH_MAX_TUNE], cand_ctas_per_sm[RH_MAX_TUNE];
    double cand_ms[RH_MAX_TUNE];       /* device time of the candidate's run */
    int64_t sample_columns;
} rh_tune_result;

int rh_autotune(rh_ctx *ctx, int32_t precision, rh_tune_result *out);

/* Copy results to host arrays (any pointer may be NULL):
 * n_out [ncol][nlev][ndep] m^-3, iters [ncol], status [ncol] (RH_COL_*),
 * dmax [ncol].  n_out may also be a device pointer when on_device = 1. */
int rh_get_populations(rh_ctx *ctx, double *n_out, int32_t *iters, uint8_t *status,
                       double *dmax, int32_t on_device);
/* LTE populations [ncol][nlev][ndep] and electron densities [ncol][ndep] (host). */
int rh_get_lte(rh_ctx *ctx, double *nstar_out, double *ne_out);
/* Set the current populations (host [ncol][nlev][ndep], finite, > 0): the
 * checkpoint / restart path (rh_iterate with start = 2). */
int rh_set_populations(rh_ctx *ctx, const double *n_in);

/* Emergent intensity I(mu, lambda) at the top of every column for the current
 * populations (Sect. 2.2: vertical emergent spectrum; mu = 1 is vertical),
 * at arbitrary wavelengths lambda_m [nlambda] (m, > 0).  I_out [ncol][nlambda]
 * in W m^-2 Hz^-1 sr^-1, host memory (on_device = 0) or device (1).
 * precision as in rh_iter_opts. */
int rh_emergent_spectrum(rh_ctx *ctx, double mu, int64_t nlambda, const double *lambda_m,
                         double *I_out, int32_t precision, int32_t on_device);

/* ---------------------------------------------------------------------- */
/* Learned initial guess.  The paper has no such start solution; it shows   */
/* that the start solution decides the iteration count (Sect. 2.3, Fig. 1) */
/* and offers LTE, zero radiation and escape probabilities.  This adds a    */
/* multilayer perceptron that maps a column's atmosphere -- T, log10 n_e,   */
/* log10 n_H and v_z at every depth, standardised -- to the log departure   */
/* coefficients ln(n_i/n*_i) at every depth.  It is trained on the GPU, on  */
/* columns that rh_iterate converged, by the library's own BF16 kernels     */
/* (tensor-core GEMMs, GELU, mean-squared error, Adam); rh_iterate with     */
/* start = 1 evaluates it and iterates from the prediction (renormalised so  */
/* that sum_i n_i = n_H) to the same convergence criterion.                  */

/* Create the network for the loaded columns' depth count: input 4 ndep,    */
/* nhidden hidden layers of `hidden` units (GELU), output nlev ndep; He-     */
/* normal weights from `seed`, zero biases.  Replaces an existing network.   */
int rh_surrogate_init(rh_ctx *ctx, int32_t hidden, int32_t nhidden, uint64_t seed);
/* Length of the network state in floats: weights and biases layer by layer */
/* (W [out][in] then b [out]), then the input means and inverse standard    */
/* deviations [4 ndep] each.  0 if no network exists.                        */
int64_t rh_surrogate_state_size(const rh_ctx *ctx);
/* Copy the state out / in (host arrays of rh_surrogate_state_size floats); */
/* setting resets the optimiser moments.  This is the checkpoint.            */
int rh_surrogate_get_state(rh_ctx *ctx, float *state_out);
int rh_surrogate_set_state(rh_ctx *ctx, const float *state_in);

typedef struct {
    int32_t epochs;          /* passes over the training columns */
    int32_t batch;           /* columns per optimiser step */
    float lr;                /* Adam learning rate (cosine-decayed over the run) */
    float beta1, beta2, eps; /* Adam constants */
    uint64_t seed;           /* shuffling */
    int32_t standardise;     /* 1: (re)compute the input standardisation on these columns */
} rh_train_opts;

typedef struct {
    double loss_first_epoch, loss_last_epoch;   /* mean squared error of ln b per epoch */
    int64_t steps, samples;
    double seconds;
} rh_train_stats;

/* Train on every loaded column whose status is RH_COL_CONVERGED (targets:  */
/* ln(n/n*) of its current populations).  RH_ESTATE without a network or   */
/* without converged columns.                                                */
int rh_surrogate_train(rh_ctx *ctx, const rh_train_opts *opts, rh_train_stats *stats_out);
/* Loss and gradient (host, rh_surrogate_state_size floats; the trailing     */
/* standardisation entries are zero) of the current network on the loaded   */
/* columns cols[0..ncols) with their current populations as targets.  For  */
/* checking the training kernels against an independent implementation.    */
int rh_surrogate_loss_grad(rh_ctx *ctx, int64_t ncols, const int32_t *cols, double *loss_out, float *grad_out);
/* Raw prediction ln(n/n*) [ncol][nlev][ndep] (host) for every loaded column. */
int rh_surrogate_predict(rh_ctx *ctx, float *lnb_out);

/* Checkpoint files of the network (host byte order, little-endian targets): */
/* "RH15DMLP", uint32 version 1, int32 nin, hidden, nhidden, nout, int64     */
/* nparam, the state (rh_surrogate_get_state's floats), and a 64-bit FNV-1a  */
/* hash of the state bytes.  save: RH_ESTATE without a network, RH_EINVAL    */
/* if the file cannot be written.  load: creates (or replaces) the network   */
/* with the file's sizes and state; RH_ESTATE without loaded columns,        */
/* RH_EINVAL for a missing, truncated or corrupted file or one made for      */
/* another depth count or atom.  file_info: checks a file without a context */
/* or GPU and returns its sizes {nin, hidden, nhidden, nout} and state       */
/* length; RH_EINVAL with the reason in msg (optional, msg_len bytes).       */
int rh_surrogate_save(rh_ctx *ctx, const char *path);
int rh_surrogate_load(rh_ctx *ctx, const char *path);
int rh_surrogate_file_info(const char *path, int32_t *sizes_out, int64_t *nparam_out, char *msg, size_t msg_len);

/* ---------------------------------------------------------------------- */
/* Shared-memory layout of the column kernel (no counterpart in the paper;  */
/* a host computation that needs no GPU, for checking the layout): the byte  */
/* offsets of its 15 regions in carve order (populations, new populations,   */
/* collisional rates, reduction scratch, rate accumulators, 3 per-depth      */
/* arrays, the per-depth background block [ndep][4], continuum factors,      */
/* damping, populations in the working precision, Voigt table, block         */
/* counters, the warps' line-profile rings) and the carve's end in           */
/* offsets_out[0..15], and the bytes the launch allocates in bytes_out (the  */
/* same function sizes and carves, so the two are equal).  macc: rate        */
/* accumulators per depth.  ring_warps (0..32): warps whose profile ring the */
/* block holds -- the block's warps for the FP32 kernel with the profile     */
/* cache and without PRD lines (2304 bytes each: three depths of up to three */
/* line profiles for the two rays of a sweep pass), 0 for the other kernels. */
/* RH_EINVAL for sizes outside the library's limits.                        */
int rh_column_smem_layout(int32_t precision, int32_t nlev, int32_t ndep, int32_t ntr, int32_t ncont, int32_t nline,
                          int32_t macc, int32_t ring_warps, size_t *offsets_out, size_t *bytes_out);

/* ---------------------------------------------------------------------- */
/* Measured fused multiply-add rate of a device (no counterpart in the      */
/* paper: the denominator of the column kernel's roofline).  precision 1    */
/* FP32, 0 FP64.  Every thread of 4 x 256-thread blocks per SM runs 16      */
/* independent chains x <- a x + b; after a calibration launch one launch   */
/* of about `seconds` (0 < seconds <= 10) is timed with CUDA events, and    */
/* flop_s_out = 2 x FMAs / its time (seconds_out, optional: that time).     */
/* Allocates a 2 KB device buffer and a stream for the call.  The caller's  */
/* current device is restored.  RH_EINVAL for bad arguments, RH_ECUDA.      */
int rh_fma_peak(int32_t device, int32_t precision, double seconds, double *flop_s_out, double *seconds_out);

/* ---------------------------------------------------------------------- */
/* rh_iterate_noalloc -- the paper has no counterpart to this call; it      */
/* exists for callers of this library that cannot allocate device memory    */
/* while they solve: programs that hand all GPU memory to their own pool or  */
/* budget (a framework allocator that must see every byte), and latency-     */
/* bound loops that cannot afford the device-wide synchronisation cudaMalloc */
/* and cudaFree imply.  Such a caller creates the context, sets the atom and */
/* loads the columns once during start-up (those calls do allocate), and     */
/* later calls this function as often as it likes.                           */
/*                                                                           */
/* It runs the same iteration as rh_iterate over every loaded column         */
/* (only_unconverged must be 0; atoms with PRD lines are refused, their      */
/* redistribution scratch is allocated).  The line profiles come from the    */
/* context's profile cache when an earlier rh_iterate or rh_solve on the     */
/* context allocated it -- the results are then bit for bit those of         */
/* rh_iterate with the same options -- and are otherwise evaluated inside    */
/* the sweep, which agrees with the cached sweep to FP32 rounding (the two   */
/* kernels' multiply-adds may be fused differently).  It writes results to  */
/* caller-owned DEVICE buffers of the context's device: n_out               */
/* [ncol][nlev][ndep] (with start = 2 it is also read as the starting       */
/* populations), iters_out [ncol], status_out [ncol] (RH_COL_*), dmax_out    */
/* [ncol].  A pointer that is not device (or managed) memory of that device  */
/* is refused with RH_EINVAL; their sizes cannot be checked here and must    */
/* hold the counts above.  It calls no cudaMalloc, cudaFree or other         */
/* allocating routine: its device scratch (work-queue counter, result       */
/* counters, the wavelength table in the iteration's precision and the Ng   */
/* history of the resident blocks) is one statically sized 9 MiB device     */
/* array inside the library, which every GPU that loads the library holds    */
/* until the process exits, and the wavelength table is staged through two   */
/* static host arrays of the library.  A problem whose Ng history for one    */
/* column exceeds the device array (4 x nlev x ndep doubles > ~8 MiB; cannot */
/* happen within the limits of rh_load_columns and rh_setup_atom) is        */
/* rejected with RH_EINVAL; a smaller array only lowers the number of        */
/* resident blocks.  The first call on each device looks the array's         */
/* address up, so make that first call before starting any stream capture.  */
/* Every call, from every context and thread, shares the device and host     */
/* arrays and keeps its counters' last contents (they are cleared at the     */
/* start of each call); calls whose GPU work overlapped would race on them.  */
/* The library holds a lock for the whole call and returns only after the    */
/* call's GPU work has finished on the context's stream, so calls from       */
/* several host threads of one process run one after another.  The caller's  */
/* current device is restored on return.  stats_out (optional, host)         */
/* reports wall-clock seconds, and max_dn_final as rh_iterate does.  Returns  */
/* RH_OK, RH_ENOTCONV, RH_EINVAL, RH_ESTATE or RH_ECUDA as rh_iterate does.   */
int rh_iterate_noalloc(rh_ctx *ctx, const rh_iter_opts *opts, double *n_out, int32_t *iters_out,
                       uint8_t *status_out, double *dmax_out, rh_iter_stats *stats_out);

#ifdef __cplusplus
}
#endif
#endif /* RH15D_H */
