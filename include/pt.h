/*
 * pt.h -- C ABI of the GB300 (sm_103a) transit-model library.
 *
 * The library evaluates the forward model of Parviainen (2015), "PyTransit:
 * fast and easy exoplanet transit modelling in Python": quadratic
 * Mandel-Agol fluxes (Sec. 2.2, Eq. ma_model) and Gimenez series fluxes
 * (Sec. 2.1, Eqs. gimenez_flux, gimenez_alpha, gimenez) over
 * time points x parameter vectors x passbands, with exposure supersampling
 * (Sec. 3.2), circular or eccentric orbits (Sec. 1), limb darkening factored
 * out of the geometry (Secs. 2.1.3, 2.2.2) and, optionally, the likelihood
 * reduction moved onto the device (Sec. 3.4).
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev / documented "device" are device (GPU) pointers,
 *     owned by the caller.  The library never frees them.  Entry points do
 *     not allocate device memory unless their comment says so (the Gimenez
 *     plan owns its coefficient tables).
 *   - `stream` is a cudaStream_t (0 = legacy default stream).  Calls are
 *     asynchronous with respect to the host: they enqueue kernels and return.
 *   - Return value: PT_OK, or a PT_ERR_* code for a host-detected error (bad
 *     size, null pointer, workspace too small, a host-side value outside its
 *     domain such as a negative exposure time) or a launch error.  The text of
 *     the last error is available from pt_last_error_string() (thread-local).
 *   - Conditions only the device can see come back through caller-provided
 *     device ints: Newton solves that hit their step cap are counted in the
 *     optional n_bad_dev of each call, and pt_domain_check() counts parameter
 *     sets outside the model's domain.  The light-curve kernels themselves do
 *     not check device-resident parameters (their results for out-of-domain
 *     values are not specified); pt_status_read() synchronises a stream and
 *     turns the two counters into PT_ERR_DOMAIN / PT_ERR_NOT_CONVERGED.
 *   - Layouts are row-major with time fastest: a flux cube is [n_v][n_b][n_t].
 *   - z of a point behind the star (the planet is not between the star and
 *     the observer) is PT_Z_BEHIND; its flux is 1.
 *
 * Readings of points the paper leaves open (repeated where they apply):
 *   - t0 is the time of inferior conjunction (true anomaly pi/2 - w).
 *   - Eccentric orbits: b = a cos i (1 - e^2)/(1 + e sin w) (Winn 2010).
 *   - Supersamples sit at t + t_exp ((s + 1/2)/n_ss - 1/2); the point value
 *     is their unweighted mean (Sec. 3.2, "n evenly distributed subsamples").
 *   - Gimenez: G_j(p,q;x) = 2F1(-j, p+j; q; x) and the series keeps
 *     j = 0 .. n_j-1 (N_J terms, Sec. 2.1.1).
 */
#ifndef PT_H
#define PT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque CUDA stream (binary-compatible with cudaStream_t). */
typedef struct CUstream_st *pt_stream_t;

enum {
    PT_OK = 0,
    PT_ERR_ARG = 1,           /* null pointer, negative size or inconsistent sizes */
    PT_ERR_DOMAIN = 2,        /* parameter outside the supported domain (host check or pt_status_read) */
    PT_ERR_NOT_CONVERGED = 3, /* Newton step cap hit (pt_status_read of an n_bad counter) */
    PT_ERR_CUDA = 4,          /* kernel launch or CUDA runtime error */
    PT_ERR_WORKSPACE = 5      /* work buffer null, misaligned or smaller than required */
};

#define PT_Z_BEHIND 1.0e30f

/* Library version (major*10000 + minor*100 + patch). */
int pt_version(void);

/* Static text of a status code. */
const char *pt_status_string(int status);

/* Text of the last CUDA error seen by this host thread ("" if none). */
const char *pt_last_error_string(void);

/*
 * Orbit parameters, structure of arrays; every array is a DEVICE pointer
 * with n_v entries.
 *   t0  : time of inferior conjunction [days]          (FP64)
 *   P   : orbital period [days]                        (FP64)
 *   a   : semi-major axis in stellar radii             (FP32)
 *   inc : inclination [radians]                        (FP32)
 *   e   : eccentricity in [0, 0.95], or NULL for circular orbits (values are not checked on the host)
 *   w   : argument of periastron [radians]; NULL iff e is NULL
 * Times are FP64 so that the phase of a point 10^3 days from t0 keeps
 * sub-millisecond accuracy; everything after the phase reduction is FP32.
 */
typedef struct pt_orbit {
    const double *t0;
    const double *P;
    const float *a;
    const float *inc;
    const float *e;
    const float *w;
    int n_v;
} pt_orbit;

/* ------------------------------------------------------------------------
 * Parameter domain and device-side status.
 *
 * pt_domain_check counts, into *n_out_dev (device int; the caller zeroes it),
 * the parameter sets outside the domain the model is defined and tested on:
 *   t0 finite; 0 < P < 1e15; 1 < a < 1e7 (the orbit lies outside the star);
 *   0 <= inc <= pi; e in [0, 0.95] and w finite when e is given;
 *   0 < k <= 1e3 (NaN fails every test).
 * k_dev holds n_k_per_v radius ratios per vector ([n_v] or [n_v][n_b]); a
 * vector counts once per failing radius ratio, plus once if its orbit fails.
 * Asynchronous on `stream`; reads its inputs only.
 *
 * pt_status_read synchronises `stream`, reads the two device counters (either
 * may be NULL) and returns PT_ERR_DOMAIN if *n_domain_dev > 0, else
 * PT_ERR_NOT_CONVERGED if *n_bad_dev > 0, else PT_OK; pt_last_error_string()
 * then gives the count.  It does not reset the counters.
 * ---------------------------------------------------------------------- */
int pt_domain_check(const pt_orbit *orb, const float *k_dev, int n_k_per_v, int *n_out_dev, pt_stream_t stream);
int pt_status_read(const int *n_bad_dev, const int *n_domain_dev, pt_stream_t stream);

/* ------------------------------------------------------------------------
 * Projected separation z(t) (Sec. 1: "circular and elliptic orbits (using
 * ... Newton's method ...)").  The paper gives no formula; the library uses
 * z = r sqrt(cos^2(w+f) + sin^2(w+f) cos^2 i), r = a(1 - e cos E), with the
 * true anomaly f from E and E from Kepler's equation E - e sin E = M.
 *
 * Output z_dev is [n_v][n_t * n_ss] (FP32): z of vector v at time index i and
 * supersample s sits at z_dev[v*n_t*n_ss + i*n_ss + s].
 * ---------------------------------------------------------------------- */

/* Circular orbit: z = a sqrt(sin^2 phi + cos^2 i cos^2 phi), phi = 2 pi (t - t0)/P
 * reduced in FP64; orb->e and orb->w are ignored. */
int pt_z_circ(const double *t_dev, int n_t, const pt_orbit *orb, int n_ss, double t_exp,
              float *z_dev, pt_stream_t stream);

/* Eccentric orbit: FP64 Newton iteration on Kepler's equation per point
 * (at most max_iter steps; converged when |dE| < tol), then z in FP32.
 * Points that did not converge are counted into *n_bad_dev (device int,
 * may be NULL; the caller zeroes it) and keep their last iterate. */
int pt_z_ecc(const double *t_dev, int n_t, const pt_orbit *orb, int n_ss, double t_exp, int max_iter,
             double tol, float *z_dev, int *n_bad_dev, pt_stream_t stream);

/* ------------------------------------------------------------------------
 * Pointwise Mandel & Agol terms (Sec. 2.2.1, Eq. ma_model; the functions
 * are those of Mandel & Agol 2002, Table 1).  For n pairs (k[i], z[i]):
 *   lam_e[i]  = uniform-disk covered fraction lambda_e,
 *   lam_d[i]  = lambda_d + 2/3 Theta(k - z)   (the Theta term folded in),
 *   eta_d[i]  = eta_d,
 * so that f = 1 - [(1-c) lam_e + c lam_d + u2 eta_d] / (1 - u1/3 - u2/6)
 * with c = u1 + 2 u2.  All FP32 device arrays; k > 0.  Any output may be NULL.
 * Accuracy: the flux formed from these terms is within 1e-6 of the FP64
 * model for k <= 1 (every tested workload has k <= 0.3).  For k > 1 the
 * brace cancels about tenfold in FP32 and the bound is 3e-6.
 * ---------------------------------------------------------------------- */
int pt_ma_terms(const float *k_dev, const float *z_dev, size_t n, float *lam_e_dev, float *lam_d_dev,
                float *eta_d_dev, pt_stream_t stream);

/* ------------------------------------------------------------------------
 * Quadratic Mandel-Agol light curves (Sec. 2.2; supersampling Sec. 3.2;
 * multiple passbands Sec. 2.2.2; device likelihood Sec. 3.4).
 *
 *   t_dev      [n_t] FP64 exposure mid-times (any order)
 *   orb        orbit parameters of the n_v vectors (circular if orb->e NULL)
 *   k_dev      radius ratios: [n_v] if k_per_band == 0, else [n_v][n_b]
 *   ld_dev     [n_v][n_b][2] quadratic coefficients (u1, u2)
 *   n_b        passbands per vector
 *   n_ss       supersamples per exposure (>= 1); t_exp exposure time [days]
 *   max_iter   cap on Newton steps for eccentric orbits, 1..64 (e.g. 16)
 *   y_dev, wt_dev  [n_b][n_t] observed fluxes and weights (wt may be NULL
 *              for unit weights); needed only when ssr_dev != NULL
 *   flux_dev   [n_v][n_b][n_t] output flux cube, or NULL
 *   ssr_dev    [n_v][n_b] output sum_t wt (y - f)^2, or NULL
 *   work_dev   device scratch of at least pt_ma_quad_work_bytes() bytes,
 *              16-byte aligned (as cudaMalloc and PyTorch allocations are;
 *              the kernels read it in 16-byte vectors)
 *   n_bad_dev  optional device int: points whose Newton iteration hit
 *              max_iter are added to it
 * With k_per_band == 0 one geometry pass serves all n_b limb-darkening sets
 * (the factoring of Sec. 2.2.2); with k_per_band == 1 every passband has its
 * own radius ratio and is evaluated as its own geometry.
 * At least one of flux_dev and ssr_dev must be non-NULL.
 * Accuracy: fluxes within 1e-6 of the FP64 model for k <= 1 (3e-6 above,
 * as for pt_ma_terms).  PT_ERR_DOMAIN for t_exp < 0 or not finite.
 * ---------------------------------------------------------------------- */
size_t pt_ma_quad_work_bytes(int n_t, int n_v, int n_b, int k_per_band);

int pt_ma_quad(const double *t_dev, int n_t, const pt_orbit *orb, const float *k_dev, int k_per_band,
               const float *ld_dev, int n_b, int n_ss, double t_exp, int max_iter, const float *y_dev,
               const float *wt_dev, float *flux_dev, float *ssr_dev, void *work_dev, size_t work_bytes,
               int *n_bad_dev, pt_stream_t stream);

/* ------------------------------------------------------------------------
 * Interpolated Mandel-Agol terms (Sec. 2.2.3).  The three functions of
 * Eq. (ma_model) are tabulated on a (k, z) grid and read back by bilinear
 * interpolation instead of being evaluated:
 *   k_i = k_lo + i (k_hi - k_lo) / (n_k - 1),   i = 0 .. n_k - 1,
 *   z_j = j (1 + k_hi) / (n_z - 1),             j = 0 .. n_z - 1
 * (z spans [0, 1 + k] for every k of the table), values
 * (lambda_e, lambda_d + 2/3 Theta(k - z), eta_d) as in pt_ma_terms, computed
 * by the exact FP32 kernel.  Reading: z >= 1 + k gives exactly zero (out of
 * transit); k outside [k_lo, k_hi] is clamped to the table's range (the
 * caller sets the range from the prior on k).  The paper's defaults are
 * n_k = 128, n_z = 256; the error against the exact model is dominated by
 * n_z (a few ppm in flux at n_z = 256).
 *
 *   pt_ma_table_create   builds the table on the device (allocates
 *                        n_k n_z 16 bytes; requires 0 < k_lo < k_hi,
 *                        2 <= n_k <= 4096, 2 <= n_z <= 65536); synchronous.
 *   pt_ma_table_destroy  frees it.
 *   pt_ma_terms_interp   pointwise drop-in for pt_ma_terms.
 *   pt_ma_quad_interp    pt_ma_quad with the interpolated terms (same
 *                        arguments, same work buffer size).
 * ---------------------------------------------------------------------- */
typedef struct pt_ma_table_s *pt_ma_table;

int pt_ma_table_create(float k_lo, float k_hi, int n_k, int n_z, pt_ma_table *table_out);
int pt_ma_table_destroy(pt_ma_table table);
int pt_ma_terms_interp(pt_ma_table table, const float *k_dev, const float *z_dev, size_t n, float *lam_e_dev,
                       float *lam_d_dev, float *eta_d_dev, pt_stream_t stream);
int pt_ma_quad_interp(pt_ma_table table, const double *t_dev, int n_t, const pt_orbit *orb, const float *k_dev,
                      int k_per_band, const float *ld_dev, int n_b, int n_ss, double t_exp, int max_iter,
                      const float *y_dev, const float *wt_dev, float *flux_dev, float *ssr_dev, void *work_dev,
                      size_t work_bytes, int *n_bad_dev, pt_stream_t stream);

/* ------------------------------------------------------------------------
 * Adjoint of the quadratic Mandel-Agol light curve (not in the paper, which
 * cites analytic MA derivatives, Pal 2008).  For n_v parameter vectors
 * theta = (t0, P, a, b, e, w, k, u1, u2), one passband, exposure times t:
 *   ssr[v]      = sum_t wt (y - f)^2,        f = mean over n_ss supersamples
 *   grad[v][i]  = d ssr[v] / d theta_i       (order t0, P, a, b, e, w, k, u1, u2)
 *   flux[v][t]  = f (optional)
 * b is the impact parameter, cos i = b (1 + e sin w) / (a (1 - e^2)).
 * The forward model is recomputed inside the kernel (no saved activations).
 * Derivatives: dF/dk and dF/dz from the moving edge of the overlap region
 * (complete elliptic integrals), then the chain rule through z, Kepler's
 * equation and the conjunction anchor.  e and w may be NULL (circular,
 * w = pi/2); their gradient entries are then d/de and d/dw at e = 0.
 * work_dev: at least pt_ma_quad_bwd_work_bytes(n_t) bytes, 16-byte aligned
 * (else PT_ERR_WORKSPACE): the double-float split of the times, and per tile
 * of 64 consecutive times (as stored in t_dev; they need not be sorted) the
 * tile's time range and its residual sum with the flux at 1,
 * sum wt (y - 1)^2, in FP64.  A tile whose range meets no transit window of
 * a vector is not evaluated for it: its flux is exactly 1 there and its
 * derivatives zero, so its residual sum is added as it stands.
 * y_dev, wt_dev: [n_t]; wt may be NULL.  ssr_dev, flux_dev may be NULL.
 * ---------------------------------------------------------------------- */
typedef struct pt_theta {
    const double *t0;
    const double *P;
    const float *a;
    const float *b;
    const float *e;
    const float *w;
    const float *k;
    const float *u1;
    const float *u2;
    int n_v;
} pt_theta;

size_t pt_ma_quad_bwd_work_bytes(int n_t);

int pt_ma_quad_bwd(const double *t_dev, int n_t, const pt_theta *theta, int n_ss, double t_exp, int max_iter,
                   const float *y_dev, const float *wt_dev, float *grad_dev, float *ssr_dev, float *flux_dev,
                   void *work_dev, size_t work_bytes, int *n_bad_dev, pt_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched evaluation for spectrophotometric MCMC (the paper's motivation,
 * Sec. 1; per-passband limb darkening and radius ratio, Secs. 2.2.2 and 3.5;
 * likelihood on the device, Sec. 3.4): n_v walkers x n_b passbands over
 * n_lc light curves of uneven length, concatenated in t.  Every passband has
 * its own k and (u1, u2); the orbit is per walker.
 *
 * pt_batch_plan_create() binds the buffers named in the descriptor (their
 * addresses, not their contents), builds a work list of (walker, time tile)
 * items that never straddle a light curve, times candidate configurations
 * (tile length 64/128/256 x CTAs per SM) on those buffers when autotune is
 * non-zero, and captures the chosen evaluation -- work-counter reset,
 * per-walker set-up, one persistent kernel, residual reduction -- into a
 * CUDA graph.  pt_batch_run() replays that graph on a stream: update the
 * contents of the bound buffers (new walker parameters, new data) between
 * runs.  The plan allocates its own work list and scratch (device memory)
 * at creation and releases them in pt_batch_plan_destroy().
 * ---------------------------------------------------------------------- */
typedef struct pt_batch_desc {
    const double *t;        /* [n_t] device, concatenated exposure times */
    int n_t;
    const int *lc_offsets;  /* [n_lc + 1] HOST: light curve j is t[lc_offsets[j] .. lc_offsets[j+1]) */
    int n_lc;
    pt_orbit orb;           /* n_v walkers (device arrays) */
    const float *k;         /* [n_v][n_b] device */
    const float *ld;        /* [n_v][n_b][2] device, (u1, u2) */
    int n_b;                /* 1..256 */
    int n_ss;               /* supersamples, 1..256 */
    double t_exp;
    int max_iter;           /* Newton cap for eccentric orbits, 1..64 */
    const float *y;         /* [n_b][n_t] device, needed with ssr */
    const float *wt;        /* [n_b][n_t] device or NULL */
    float *flux;            /* [n_v][n_b][n_t] device or NULL */
    float *ssr;             /* [n_v][n_b] device or NULL (not both NULL) */
    int *n_bad;             /* optional device counter of non-converged Newton solves */
    int k_mode;             /* 0: each passband with its own k (exact);
                               1: the model once per walker with k_hat, the mean of its
                                  passbands' k, and each passband's depth 1 - f scaled by
                                  k_b^2 / k_hat^2 (Sec. 3.5);
                               2: each passband with its own k, the Mandel-Agol terms read
                                  from `table` by bilinear interpolation in (k, z)
                                  (Sec. 2.2.3; k outside the table's range is clamped) */
    pt_ma_table table;      /* k_mode 2: a table of pt_ma_table_create, owned by the caller
                               and kept alive while the plan runs; NULL otherwise */
} pt_batch_desc;

typedef struct pt_batch_plan_s *pt_batch_plan;

int pt_batch_plan_create(const pt_batch_desc *desc, int autotune, pt_batch_plan *plan_out);
int pt_batch_run(pt_batch_plan plan, pt_stream_t stream);
int pt_batch_plan_info(pt_batch_plan plan, int *tile, int *ctas_per_sm, int *n_items, float *tuned_ms);
int pt_batch_plan_destroy(pt_batch_plan plan);

/* ------------------------------------------------------------------------
 * Surrogate network for the ingress/egress Mandel-Agol terms (not in the
 * paper; its analogue there is the interpolation tables of Sec. 2.2.3).
 * A multilayer perceptron 2 -> 128 -> 128 -> 128 -> 2 with SiLU
 * activations, silu(x) = x / (1 + exp(-x)), maps normalised (k, s) to
 * normalised (lambda_d / k^2, eta_d / k^2) over the ingress/egress band
 * z = |1 - k| + 2 min(k, 1) s, s in [0, 1].  Parameters (FP32, device),
 * flattened:  W1[128][2] b1[128] W2[128][128] b2[128] W3[128][128] b3[128]
 * W4[2][128] b4[2].
 *
 * Training entry points (FP32 SIMT kernels):
 *   pt_sur_datagen     n samples (k, s) from a counter-based generator
 *                      (splitmix64 of seed and index offset..offset+n-1),
 *                      targets from the exact FP32 kernel, written as
 *                      X[n][2] = ((k - norm[0])/norm[1], (2/pi) acos(1 - 2s) - 1),
 *                      T[n][2] = ((ld/k^2 - norm[2])/norm[3], (ed/k^2 - norm[4])/norm[5]),
 *                      kz[n][2] = (k, z); X, T or kz may be NULL (not all)
 *   pt_mlp_forward     Y[n][2] for inputs X (FP32 reference forward; qat as below)
 *   pt_mlp_loss_grad   loss = mean_i sum_o (y - t)^2 and its gradient; with
 *                      qat != 0 the tensor-core layers' operands (h1, h2,
 *                      W2, W3) are rounded to BF16 in the forward pass, as
 *                      inference serves them (straight-through gradient)
 *   pt_mlp_adam        one Adam step (bias-corrected, step >= 1)
 * work: pt_mlp_work_bytes(n).  Reductions are deterministic.
 * ---------------------------------------------------------------------- */
#define PT_MLP_HIDDEN 128
#define PT_MLP_NPARAMS 33666

size_t pt_mlp_work_bytes(int n);
int pt_sur_datagen(unsigned long long seed, size_t offset, size_t n, float k_lo, float k_hi, const float *norm_dev,
                   float *X_dev, float *T_dev, float *kz_dev, pt_stream_t stream);
int pt_mlp_forward(const float *params_dev, const float *X_dev, int n, int qat, float *Y_dev, void *work_dev,
                   size_t work_bytes, pt_stream_t stream);
int pt_mlp_loss_grad(const float *params_dev, const float *X_dev, const float *T_dev, int n, int qat,
                     float *grad_dev, float *loss_dev, void *work_dev, size_t work_bytes, pt_stream_t stream);
int pt_mlp_adam(float *params_dev, const float *grad_dev, float *m_dev, float *v_dev, int step, float lr,
                float beta1, float beta2, float eps, pt_stream_t stream);

/* Serving the surrogate (BF16 tensor cores, tcgen05.mma, FP32 accumulation):
 *   pt_sur_model_create  copies FP32 parameters (device), packs W2 and W3 to
 *                        BF16 in the tensor-core operand layout, and keeps
 *                        the normalisation (norm[6] as in pt_sur_datagen), the
 *                        k range of the band and an error-bound table
 *                        (host, [nk][ns] over k in [k_lo, k_hi] x s in [0,1);
 *                        1 = use the exact kernel in that cell).  Allocates
 *                        device memory; pt_sur_model_destroy frees it.
 *   pt_ma_surrogate      drop-in for pt_ma_terms: (lambda_e, lambda_d + 2/3
 *                        Theta(k - z), eta_d) for n pairs (k, z).  Points in
 *                        the band and in unmarked cells take lambda_d and
 *                        eta_d from the network (lambda_e exact); all others
 *                        take the exact FP32 kernel (computed while the points
 *                        are classified) and are counted in *n_fallback_dev
 *                        (optional device int, caller zeroes it); the
 *                        network's points are compacted into a list in
 *                        work_dev (pt_sur_work_bytes(n) bytes).
 *   pt_sur_mlp_eval      raw network outputs Y[n][2] for normalised inputs
 *                        X[n][2] on the tensor-core path.
 *   pt_sur_cell_errors   per-cell maximum over points of
 *                        4 |ld_sur - ld_ref| + 2 |ed_sur - ed_ref| (a bound of
 *                        the flux error for q1, q2 in [0, 1]), atomically
 *                        maxed into cell_max[nk][ns] (caller zeroes it).
 *   pt_sur_model_error   1 if a tensor-core wait ever timed out (the kernel
 *                        then skipped its remaining tiles), else 0.
 * ---------------------------------------------------------------------- */
typedef struct pt_sur_model_s *pt_sur_model;

int pt_sur_model_create(const float *params_dev, const float *norm, float k_lo, float k_hi,
                        const unsigned char *table, int nk, int ns, pt_sur_model *model_out);
int pt_sur_model_destroy(pt_sur_model model);
size_t pt_sur_work_bytes(size_t n);
int pt_ma_surrogate(pt_sur_model model, const float *k_dev, const float *z_dev, size_t n, float *lam_e_dev,
                    float *lam_d_dev, float *eta_d_dev, int *n_fallback_dev, void *work_dev, size_t work_bytes,
                    pt_stream_t stream);
int pt_sur_mlp_eval(pt_sur_model model, const float *X_dev, size_t n, float *Y_dev, pt_stream_t stream);
int pt_sur_cell_errors(const float *k_dev, const float *z_dev, const float *ld_ref_dev, const float *ed_ref_dev,
                       const float *ld_sur_dev, const float *ed_sur_dev, size_t n, float k_lo, float k_hi, int nk,
                       int ns, float *cell_max_dev, pt_stream_t stream);
int pt_sur_model_error(pt_sur_model model, int *err_host);

/* ------------------------------------------------------------------------
 * pt_ma_quad without a work buffer.  The paper has no counterpart: this is
 * an interface for callers that cannot allocate device memory -- e.g. a host
 * program whose device memory is all owned by its own fixed pool, or a tight
 * sampling loop that must not stall on an allocation.  Arguments and results
 * are those of pt_ma_quad minus work_dev/work_bytes; the caller still owns
 * every input and output.
 *
 * Scratch comes from a static device array of PT_MA_NOALLOC_SCRATCH_BYTES
 * (4 MiB) that every GPU loading the library keeps until the process exits.
 * The call runs the tile kernel, whose scratch is, with each term rounded up
 * to a multiple of 256 bytes,
 *   96 n_geom + 8 n_t + 4 n_v n_b ceil(n_t / 256)
 * (n_geom = n_v, or n_v n_b with k_per_band); this is less than
 * pt_ma_quad_work_bytes(), which sizes pt_ma_quad's pair lists.  A problem
 * above the limit is rejected with PT_ERR_WORKSPACE (see
 * pt_last_error_string()): for one passband that is about n_t > 375,000 at
 * 200 vectors, or n_t > 173,000 at 1,000.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The call allocates and frees nothing.
 * All calls share the one array and it keeps the last call's contents;
 * each call writes every scratch byte it reads, so nothing needs clearing,
 * but calls that overlap on the GPU (different streams or threads) race on
 * it and must be serialised by the caller.
 * ---------------------------------------------------------------------- */
#define PT_MA_NOALLOC_SCRATCH_BYTES (4u << 20)

int pt_ma_quad_noalloc(const double *t_dev, int n_t, const pt_orbit *orb, const float *k_dev, int k_per_band,
                       const float *ld_dev, int n_b, int n_ss, double t_exp, int max_iter, const float *y_dev,
                       const float *wt_dev, float *flux_dev, float *ssr_dev, int *n_bad_dev,
                       pt_stream_t stream);

/* ------------------------------------------------------------------------
 * Gimenez series light curves (Sec. 2.1).
 *
 * A plan holds the tables of Sec. 2.1.4 for a given number of general-law
 * coefficients N (Eq. ld_general; alpha_0..alpha_N are evaluated) and series
 * depth n_j: the recursion coefficients of G_j(nu+2, 1; x) and the A_{n,j}
 * of Eq. (gimemez_a), in device memory allocated by pt_gim_plan_create and
 * released by pt_gim_plan_destroy.  1 <= N <= 16, 2 <= n_j <= 512.
 * A plan may be used from any stream; its tables are read-only after
 * creation.  The plan also owns a CUDA stream (the device's highest priority)
 * and two events: pt_gimenez forks the per-geometry table recursion and the
 * series coefficients, which depend on k alone, onto that stream at the start
 * of the call (after all earlier work of the call's stream) and joins it
 * before the evaluation kernel, so that they run beside the set-up and window
 * kernels.  Calls from several host threads or streams may share a plan:
 * their forked work runs in the order the calls were made.  Stream capture of
 * a call captures the fork and the join.
 * ---------------------------------------------------------------------- */
typedef struct pt_gim_plan_s *pt_gim_plan;

int pt_gim_plan_create(int N, int n_j, pt_gim_plan *plan_out);
int pt_gim_plan_destroy(pt_gim_plan plan);

/* Profiling hook: ev_start and ev_end (cudaEvent_t handles, owned by the
 * caller, which keeps them alive while calls use them) are recorded on the
 * call's stream right before and right after the series-evaluation kernel
 * of every later pt_gimenez call with this plan, so that the caller can time
 * that kernel alone; NULL, NULL stops it.  This is the one setting that
 * changes a plan: a plan with events set must not be used by two host
 * threads at once.  PT_ERR_ARG for a NULL plan or exactly one NULL event. */
int pt_gim_plan_time_evaluation(pt_gim_plan plan, void *ev_start, void *ev_end);

/* Pointwise alpha_n (Eq. gimenez): alpha_dev is [n][N+1] for n pairs (k, z). */
int pt_gimenez_alpha(pt_gim_plan plan, const float *k_dev, const float *z_dev, size_t n,
                     float *alpha_dev, pt_stream_t stream);

/* Light curves: arguments as pt_ma_quad, with ld_dev [n_v][n_b][N] holding
 * u_1..u_N of Eq. (ld_general) and f = 1 - sum_n C_n alpha_n (Sec. 2.1.3). */
size_t pt_gimenez_work_bytes(pt_gim_plan plan, int n_t, int n_v, int n_b, int k_per_band);

int pt_gimenez(pt_gim_plan plan, const double *t_dev, int n_t, const pt_orbit *orb, const float *k_dev,
               int k_per_band, const float *ld_dev, int n_b, int n_ss, double t_exp, int max_iter,
               const float *y_dev, const float *wt_dev, float *flux_dev, float *ssr_dev, void *work_dev,
               size_t work_bytes, int *n_bad_dev, pt_stream_t stream);

/* ------------------------------------------------------------------------
 * Gimenez light curves interpolated in z (Sec. 3.3).  Per geometry,
 * alpha_0 .. alpha_N are evaluated on n_in points over z in [0, zb],
 * zb = max(1 - k, 0), and n_edge points over (zb, 1 + k]:
 *   z_i = i zb / (n_in - 1),  i < n_in;   z_{n_in + j} = zb + (j + 1)(1 + k - zb) / n_edge,
 * and every (time, supersample) reads them by linear interpolation (zero
 * out of transit).  The flux is linear in alpha_n, so this equals
 * interpolating each passband's flux.  Arguments, outputs and errors are
 * those of pt_gimenez, plus the grid; work_dev needs
 * pt_gimenez_zi_work_bytes() bytes.  Requires n_in >= 2, n_edge >= 1 and
 * (n_in + n_edge)(N + 1) <= 16384.  At n_in = n_edge = 64 the flux error
 * against pt_gimenez is ~10-25 ppm at most (first order in the grid near
 * z = k, where alpha_n has a kink; second order elsewhere).
 * ---------------------------------------------------------------------- */
size_t pt_gimenez_zi_work_bytes(pt_gim_plan plan, int n_in, int n_edge, int n_t, int n_v, int n_b, int k_per_band);

int pt_gimenez_zi(pt_gim_plan plan, int n_in, int n_edge, const double *t_dev, int n_t, const pt_orbit *orb,
                  const float *k_dev, int k_per_band, const float *ld_dev, int n_b, int n_ss, double t_exp,
                  int max_iter, const float *y_dev, const float *wt_dev, float *flux_dev, float *ssr_dev,
                  void *work_dev, size_t work_bytes, int *n_bad_dev, pt_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* PT_H */
