/*
 * librd: forward / adjoint / gradient / Gauss-Newton Hessian-vector solve of
 * the tumor reaction-diffusion model
 *
 *     dc/dt = div(kappa(x) grad c) + rho(x) c (1 - c)      in [0, 2 pi)^3 x (0, 1]
 *     c(0)  = Phi p = sum_i p_i exp(-|x - x_i|^2 / (2 sigma^2))
 *     kappa = k_f sum_i k_i m_i,   rho = rho_f sum_i rho_i m_i
 *
 * (Scheufele et al., "Image-driven biophysical tumor growth model
 * calibration": state equation Eq. tumor:fwd and tumor:fwd-init, coefficients
 * Eq. coeff_tumor, adjoint Eq. tumor:adj / tumor:adj-final, gradients Eq.
 * tumor:inv and tumor:inv_diff, discretisation Sec. 3.3: Fourier
 * pseudo-spectral derivatives on a periodic grid, second-order Strang
 * splitting with the exact logistic reaction step and Crank-Nicolson
 * diffusion).  The Crank-Nicolson system (I - tau/2 A) x = b is solved by
 * preconditioned CG with the spectral constant-coefficient preconditioner
 * 1 / (1 + tau/2 * kbar * |k|^2), kbar the mean of kappa over the voxels
 * where it is positive.
 *
 * Plain C ABI: host or device pointers and sizes only.  One context drives
 * one grid on the current CUDA device and one stream.
 *
 * Conventions
 *   - Grid n[0] x n[1] x n[2], n[2] fastest (C order); point i of an axis of
 *     length n sits at x = 2 pi i / n.  Each n[a] must be one of
 *     8, 16, 32, 64, 96, 128, 256 (RD_ERR_SHAPE otherwise; 96 = 3 * 32 uses a
 *     radix-3 stage).
 *   - Every field passed in or out is FP64 and may live in host or device
 *     memory (unified addressing decides); it is only read (or written)
 *     during the call, the library keeps its own copy.
 *   - Parameter vectors (p, v, gradients) are FP64 host arrays of length
 *     np + 2 laid out [p_1 .. p_np, k_f, rho_f] where a full vector is meant.
 *   - Misfit J = 1/2 h^3 sum_x (c(1) - d)^2 + 1/2 beta_p |p|^2 with
 *     h^3 = (2 pi)^3 / (n0 n1 n2) (the L2 quadrature of D_c, Table 1).
 *   - Adjoint convention: alpha(1) = d - c(1) (Eq. tumor:adj-final).
 *   - Errors are returned as status codes; a call never aborts the process.
 *     rd_last_error() gives a message.  RD_ERR_NOCONV means some PCG solve
 *     hit pcg_maxit; results are still written.  RD_ERR_NONFINITE means a
 *     NaN or Inf reached a solver reduction (from the tissue maps or the
 *     data); the context stays usable once the inputs are replaced.
 *   - Argument checks happen before any launch (RD_ERR_ARG): field pointers
 *     must be non-null and 8-byte aligned; p, v, k_f, rho_f must be finite
 *     and k_f >= 0.
 *   - A context is not thread safe.  Calls are ordered on its stream; calls
 *     returning host values (rd_gradient, rd_hessvec, rd_forward with a
 *     misfit) synchronise that stream.
 */
#ifndef RD_H
#define RD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rd_ctx rd_ctx;

typedef enum {
  RD_OK = 0,
  RD_ERR_ARG = 1,        /* null pointer or out-of-range argument           */
  RD_ERR_SHAPE = 2,      /* unsupported grid size                           */
  RD_ERR_CUDA = 3,       /* a CUDA call failed (message in rd_last_error)   */
  RD_ERR_NOMEM = 4,      /* workspace too small / allocation failed         */
  RD_ERR_NOCONV = 5,     /* a PCG solve reached pcg_maxit                   */
  RD_ERR_NONFINITE = 6,  /* a NaN or Inf appeared in a reduction            */
  RD_ERR_STATE = 7       /* a required rd_set_* call has not been made      */
} rd_status;

typedef enum { RD_FP64 = 0, RD_MIXED = 1 } rd_precision;

typedef struct {
  int n[3];          /* grid                                                 */
  int nt;            /* time steps to t_end                                  */
  double t_end;      /* final time (1.0 in the normalised model)             */
  int prec;          /* RD_FP64: all FP64.  RD_MIXED: fields in FP32,
                        reductions, norms and scalars in FP64               */
  double pcg_rtol;   /* state and adjoint solves stop when ||r|| <= pcg_rtol ||b||,
                        b the right-hand side of the Crank-Nicolson system;
                        tangent-linear solves when ||r|| <= pcg_rtol ||f|| (f: rhs of the
                        increment system (I - tau/2 A) dx = f, dx0 = 0)      */
  int pcg_maxit;
  int ckpt_stride;   /* 0: keep every step's state for the adjoint;
                        s > 0: keep every s-th state and recompute segments  */
  double k_w[3];     /* k_i of Eq. coeff_tumor (WM, GM, CSF)                */
  double rho_w[3];   /* rho_i of Eq. coeff_tumor                            */
  double beta_p;     /* weight of 1/2 |p|^2 in the objective                 */
  int moving_atlas;  /* 1: reserve fields for the Moving-Atlas anatomy misfit
                        (rd_set_anatomy_data); 0: tumor misfit only          */
  int coupling;      /* 1: keep the per-voxel adjoint integrands for
                        rd_coupling_field (two more fields); 0: off          */
  int guess_restart; /* initial guesses of the state solves.  Each state solve
                        starts from the increments of the two previous steps,
                        extrapolated linearly in time (one previous step:
                        that increment), with the residual formed from their
                        stored images under (I - tau/2 A), so no operator is
                        applied.  The extrapolation restarts from a zero
                        guess at step 0, at every step that is a multiple of
                        guess_restart (> 0) and, with ckpt_stride, at every
                        segment start, so that a recomputed segment repeats
                        the forward run bit for bit (a store-all run with
                        guess_restart = ckpt_stride gives the same bits).
                        -1: every state solve starts from zero.  The solves
                        stop by the same rule either way.  Default 0.        */
} rd_config;

/* Fill *cfg with defaults: 64^3, nt 16, t_end 1, FP64, rtol 1e-10, maxit
 * 200, store all steps, k = (1, 0.1, 0), rho = (1, 0.2, 0), beta_p 0,
 * extrapolated state-solve guesses restarting only at step 0. */
rd_status rd_config_default(rd_config* cfg);

/* Device workspace in bytes that rd_create needs for cfg and np Gaussians. */
rd_status rd_workspace_size(const rd_config* cfg, int np, size_t* bytes);

/* Create a context.  workspace: device memory of at least
 * rd_workspace_size() bytes, 256-byte aligned, owned by the caller and kept
 * alive until rd_destroy; NULL makes the library allocate (and free) it.
 * stream: a cudaStream_t (NULL = legacy default stream). */
rd_status rd_create(rd_ctx** out, const rd_config* cfg, int np, void* workspace,
                    size_t workspace_bytes, void* stream);

/* Tissue probability maps m_WM, m_GM, m_CSF (Sec. 2 notation), FP64, each
 * n0 n1 n2 values; kappa1 = sum k_i m_i and rho1 = sum rho_i m_i are formed
 * on the device (Eq. coeff_tumor). */
rd_status rd_set_tissue(rd_ctx* ctx, const double* m_wm, const double* m_gm, const double* m_csf);

/* Gaussian basis (Eq. tumor:fwd-init): centers is a host array [np][3] in
 * box coordinates, sigma the common width.  Minimum-image distance. */
rd_status rd_set_basis(rd_ctx* ctx, const double* centers, double sigma);

/* Target data d (FP64 field) for the misfit. */
rd_status rd_set_data(rd_ctx* ctx, const double* d);

/* Moving-Atlas objective (Eq. objective_tu): patient anatomy labels
 * m_D = (m_D,WM, m_D,GM, m_D,CSF), FP64 fields, host or device.  Needs
 * cfg.moving_atlas = 1.  From then on the misfit is
 * D_c + D_m = 1/2 h^3 sum (c(1) - d)^2 + 1/2 h^3 sum_i sum (m_i (1 - c(1)) - m_D,i)^2
 * with m the tissue maps of rd_set_tissue, the adjoint final condition is
 * alpha(1) = d - c(1) + m^T (m (1 - c(1)) - m_D) (Eq. tumor:adj-final), and
 * rd_hessvec weights the tangent c(1) by 1 + sum_i m_i^2. */
rd_status rd_set_anatomy_data(rd_ctx* ctx, const double* md_wm, const double* md_gm, const double* md_csf);

/* Picard coupling field of the registration step (Sec. 2.2):
 *   q_i(x) = int_0^1 kbar_i grad c . grad alpha + rhobar_i c (1 - c) alpha dt,
 * kbar = k_f k_w, rhobar = rho_f rho_w, for the (p, k_f, rho_f) of the last
 * rd_gradient / rd_adjoint / rd_batch_gradient, with the time quadrature
 * of the discrete gradient and the sign of a derivative: a change dm of the
 * tissue maps inside the coefficients (Eq. coeff_tumor) changes the
 * objective by h^3 sum_x sum_i q_i dm_i at first order.  Writes three FP64
 * fields (host or device, n0*n1*n2 each, z fastest).  Needs cfg.coupling = 1;
 * RD_ERR_STATE before a gradient or after anything that invalidates it
 * (a later rd_forward, or rd_hessvec at other parameters, new tissue, data
 * or anatomy data). */
rd_status rd_coupling_field(rd_ctx* ctx, double* q_wm, double* q_gm, double* q_csf);

/* State solve (Eq. tumor:fwd): c(1) for parameters (p, k_f, rho_f); p is a
 * host array of np values.  c1_out (FP64 field, may be NULL) receives c(1);
 * misfit (host, may be NULL) receives J if data are set. */
rd_status rd_forward(rd_ctx* ctx, const double* p, double k_f, double rho_f, double* c1_out,
                     double* misfit);

/* Adjoint solve (Eq. tumor:adj) for the last rd_forward: alpha(0) into
 * alpha0_out (FP64 field, may be NULL); the reduced gradient of that point
 * is kept and can be read with rd_last_gradient. */
rd_status rd_adjoint(rd_ctx* ctx, double* alpha0_out);

/* Misfit and reduced gradient [g_p (np), g_kf, g_rhof] (Eq. tumor:inv,
 * tumor:inv_diff and the rho_f analogue) at (p, k_f, rho_f).  grad is a
 * host array of np + 2 values.  Synchronises. */
rd_status rd_gradient(rd_ctx* ctx, const double* p, double k_f, double rho_f, double* misfit,
                      double* grad);

/* Gradient of the last rd_adjoint / rd_gradient call (host, np + 2). */
rd_status rd_last_gradient(const rd_ctx* ctx, double* grad);

/* Gauss-Newton Hessian-vector product H v = J^T (h^3 J v) + beta_p v_p with
 * J = d c(1) / d(p, k_f, rho_f), from the tangent-linear model and the
 * adjoint of the same discretisation.  v and Hv: host, np + 2.
 * Synchronises. */
rd_status rd_hessvec(rd_ctx* ctx, const double* p, double k_f, double rho_f, const double* v,
                     double* Hv);

/* Reduced gradients of `count` independent problems -- each its own
 * context, grid size (uneven sizes allowed), coefficients and data -- in ONE
 * CUDA-graph launch (config "batched forward + adjoint": many parameter sets
 * or subjects at once).  The graph has one branch per context; inside a
 * branch every PCG solve is a device-side WHILE node, so the batch runs with
 * no host round trip.  p[i] (host, np_i values), k_f[i], rho_f[i] are the
 * parameters of problem i; misfit[i] (may be NULL) and grad[i] (host, np_i
 * + 2 values) receive what rd_gradient would return.  The first call for a
 * list of contexts runs one ordinary gradient on every context that has not
 * run yet, then captures the graph; later calls with the same list (same
 * order) replay it with the new parameters.  Contexts may not repeat.
 * Synchronises every context's stream before and the batch after. */
rd_status rd_batch_gradient(rd_ctx* const* ctxs, int count, const double* const* p, const double* k_f,
                            const double* rho_f, double* misfit, double* const* grad);

/* Building blocks, exposed for testing and for callers composing their own
 * solvers.  Au = k_f div(kappa1 grad u) with the Fourier pseudo-spectral
 * derivatives of Sec. 3.3 (i k zeroed at the Nyquist index); z = M^-1 r with
 * M^-1 = F^-1 diag(1 / (1 + tau/2 k_f kbar1 |k|^2)) F (kbar1 the mean of
 * kappa1 where it is positive), the PCG
 * preconditioner.  Fields FP64, host or device; needs rd_set_tissue. */
rd_status rd_apply_operator(rd_ctx* ctx, double k_f, const double* u, double* Au);

/* Tuning of the PCG preconditioner (this implementation's choice; the paper
 * names no preconditioner): kbar1 := scale * (mean of kappa1 over the
 * voxels where it is positive).  Default 1; kept across rd_set_tissue.
 * Changes only the convergence of the PCG solves, not what they converge
 * to.  RD_ERR_ARG unless scale > 0 and finite. */
rd_status rd_set_precond_scale(rd_ctx* ctx, double scale);
rd_status rd_apply_precond(rd_ctx* ctx, double k_f, const double* r, double* z);

/* Allocation-free preconditioner application (the paper has no counterpart;
 * it exists for callers that cannot allocate device memory where they need
 * it: applications whose device memory belongs to another framework's pool,
 * and latency-critical loops that must not pay cudaMalloc's implicit device
 * synchronisation).  Computes z = F^-1 [F r / (1 + coef |k~|^2)] (the PCG
 * preconditioner above with coef = tau/2 k_f kbar1) for FP64 device
 * fields r and z on grid n[0] x n[1] x n[2] (each a power of two from 8 to 256,
 * or 96;
 * RD_ERR_SHAPE otherwise), ordered on `stream`.  No context, no workspace: the
 * solver scalars, reduction partials and twiddle tables live in one fixed
 * 128 KiB __device__ array of the library, held by every GPU that loads it
 * until exit.  The first call on a device finds that array's address and
 * uploads the tables (synchronously); make that first call before any stream
 * capture.  All calls share the array, so calls that overlap on the GPU race;
 * order them on one stream.  Each call starts by clearing the array's solver
 * state and counters on `stream`, so nothing of an earlier call is read.
 * coef must be finite and >= 0; r is not modified; z may not alias r; both
 * must be 16-byte aligned (RD_ERR_ARG otherwise).  The passes' device-side
 * waits are bounded; if one gives up, z is left incomplete and this entry
 * point, having no status buffer of the caller's, cannot report it. */
rd_status rd_apply_precond_static(const int n[3], double coef, const double* r, double* z, void* stream);

/* Counters of the last call: PCG iterations summed over its solves, and
 * the number of solves. */
int rd_last_pcg_iters(const rd_ctx* ctx);
int rd_last_pcg_solves(const rd_ctx* ctx);
/* Of those solves, how many ran as a CUDA graph (device-side iteration loop)
 * rather than host-driven; host-driven solves are the first two of a
 * context and every solve while launch timing is on. */
int rd_last_graph_solves(const rd_ctx* ctx);

/* Optional launch timing, process wide.  rd_profile_enable(1) clears the
 * totals and brackets every kernel launch with two CUDA events on its stream;
 * rd_profile_read waits for the recorded events and fills, per kernel class
 * (names from rd_profile_class), the summed device milliseconds and the
 * launch counts; it returns the number of classes. */
void rd_profile_enable(int on);
int rd_profile_read(double* ms, long long* launches, int n);
const char* rd_profile_class(int i);

/* Autotuner (no counterpart in the paper): on this context's grid, time
 * `reps` PCG iterations for every candidate of each kernel class of the PCG
 * loop and keep the fastest, per kernel class and pencil length.  Candidates
 * are the tile shape -- the TMA tile kernel (64-byte column tiles along the
 * strided axes, whole-row tiles along the contiguous one, staged in shared
 * memory) or the pencil kernel (256-thread blocks of pencil groups with
 * direct loads) -- times the persistent grid size (all resident blocks, or
 * 1..8 blocks per SM).  The choice applies to every later launch in the
 * process for that class and length, so contexts of other grid sizes keep
 * their own.  caps / pencil (may be NULL) receive, for the first ncaps
 * classes of rd_profile_class, the chosen block count (0 = all resident
 * blocks) and tile shape (1 = pencil kernel) for this grid's contiguous-axis
 * length.  Leaves the PCG work fields modified (not the state, data or
 * trajectory). */
rd_status rd_autotune(rd_ctx* ctx, int reps, int* caps, int* pencil, int ncaps);
/* Forget every autotuner choice (back to TMA tiles and all resident blocks). */
void rd_autotune_clear(void);

/* Message of the last failing call ("" if none). */
/* Self-test of the bounded device-side wait that every TMA pass uses (no
 * counterpart in the paper; it lets a test reach the timeout path without
 * hanging anything).  One block arms an mbarrier for a 16-byte transaction
 * and, if copy != 0, issues a 16-byte bulk copy from src16 (device, 16-byte
 * aligned) that completes it; it then waits with at most `polls` polls
 * (1 .. the passes' own limit, 2^26) and writes to *status (device int,
 * 4-byte aligned): 0 when the wait completed and the copied bytes match, 7
 * (the timeout code that the passes record, reported as RD_ERR_CUDA "a TMA
 * wait timed out") when it gave up, -1 when the copied bytes differ.
 * Asynchronous on `stream`; RD_ERR_ARG for bad arguments. */
rd_status rd_selftest_bounded_wait(unsigned polls, int copy, const void* src16, int* status, void* stream);

/* Work actually done by the operator passes: after rd_set_tissue, counts[0..5]
 * = (active, all) tiles of the axis-0 strided passes, the axis-1 strided
 * passes and the contiguous-axis row tiles.  A tile is active when kappa1 is
 * not identically zero on it; the operator d_a(kappa d_a u) and the k_f
 * integrand vanish exactly on the others (kappa = 0 outside the brain,
 * Sec. 2.1), so the passes skip them.  RD_ERR_STATE before rd_set_tissue. */
rd_status rd_active_tiles(const rd_ctx* ctx, long long* counts);

/* Hardware probe (no counterpart in the paper): the fused multiply-add rate
 * of the current device in TFLOP/s (2 flops per FMA), FP64 for RD_FP64 and
 * FP32 for RD_MIXED, from a register-only FMA loop over every SM timed with
 * CUDA events.  It places the FP64 path, whose FFT passes do ~2-6 flops per
 * byte, on the arithmetic roofline.  Allocates and frees a small output
 * buffer; synchronous. */
rd_status rd_probe_fma_rate(int prec, double* tflops);

const char* rd_last_error(const rd_ctx* ctx);

/* Release the context (and the workspace if the library allocated it). */
void rd_destroy(rd_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* RD_H */
