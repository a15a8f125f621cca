/*
 * fp.h -- C ABI of the GB300 batched Neel-rotation Fokker-Planck library (libfp.so).
 *
 * The library computes, for many independent instances, the mean magnetic
 * moment of an ensemble of immobilised, uniaxially anisotropic nanoparticles
 * under an MPI drive field, and the normalised induced-voltage signal:
 *
 *   Eq. mean_magmom_FP (Sec. 2.1):  m_bar(t) = m0 * integral_{S^2} m f(m, t) dm
 *   Eq. FP-general     (Sec. 2.1):  df/dt = div(1/(2 tau) grad f) - div(b f)
 *   Eq. convection     (Sec. 2.1):  b = p1 H x m + p2 (m x H) x m
 *                                       + p3 (n.m) n x m + p4 (n.m) (m x n) x m
 *   Neel constants     (Sec. 2.1):  p1 = g mu0, p2 = g alpha mu0, p3 = 2 g K/Ms,
 *                                   p4 = alpha p3, tau = V Ms / (2 kB T g alpha),
 *                                   g = gamma / (1 + alpha^2), V = pi d^3 / 6
 *   Applied field      (Sec. 2):    H(r, t) = H_SF(r) + H_DF(t); the PDE has no
 *                                   r-derivative, so each voxel offset is an
 *                                   independent instance (Sec. 2.1, last paragraph)
 *   Signal             (Sec. 2.2):  phi_hat_k = 1/(m0 T) int_0^T p . dm_bar/dt
 *                                   exp(-2 pi i t k / T) dt   (model M1)
 *
 * Units: SI, with every magnetic field given as B = mu0 H in tesla (the paper
 * writes fields in T/mu0), so mu0 never enters.  Angles in radians; the easy
 * axis is n = (sin theta cos phi, sin theta sin phi, cos theta); the paper's
 * in-plane angle vartheta (Sec. 2.2 (iii)) is theta = pi/2, phi = vartheta.
 *
 * Discretisation: real spherical-harmonic Galerkin expansion of f truncated at
 * degree L (N = (L+1)^2 coefficients), the operator applied matrix-free from
 * closed-form coupling coefficients in the easy-axis frame.  Time integration:
 * Radau IIA (3 stages, order 5, or 5 stages, order 9; L-stable) with per-instance adaptive steps,
 * simplified Newton iterations whose residuals are FP64 and whose iteration
 * matrices are factorised in FP32.  Initial state: Boltzmann equilibrium at
 * H(0) including the anisotropy.
 *
 * Conventions for every entry point:
 *   - return 0 on success, a negative FP_E* code on argument or CUDA error;
 *     fp_last_error() then holds a one-line message (thread-local);
 *   - "d_" pointers are DEVICE pointers owned by the caller; "h_" pointers are
 *     host pointers owned by the caller; the library keeps none of them;
 *   - calls with a stream argument are asynchronous on that stream
 *     (cudaStream_t passed as void*, NULL = legacy default stream);
 *   - the context owns only its coefficient tables and constants (allocated
 *     once in fp_setup) and is not thread-safe: one host thread per context.
 */
#ifndef FP_H_
#define FP_H_

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes (return values) ---------------------------------------- */
#define FP_OK            0
#define FP_EINVAL       -1   /* bad argument (NULL, size, range)               */
#define FP_ECUDA        -2   /* a CUDA runtime call failed                     */
#define FP_ENOMEM       -3   /* host or device allocation failed (fp_setup)    */
#define FP_EUNSUPPORTED -4   /* valid request outside what the library supports  */

/* ---- per-instance status codes (d_status) ------------------------------- */
#define FP_STATUS_OK             0
#define FP_STATUS_MAXSTEPS       1  /* step budget (fp_tol.max_steps) exhausted */
#define FP_STATUS_STEP_UNDERFLOW 2  /* step size fell below 1e-6 of the sample spacing */
#define FP_STATUS_NONFINITE      3  /* NaN/Inf in the state                      */
#define FP_STATUS_NEWTON_FAIL    4  /* Newton iteration failed at the minimum step */
#define FP_STATUS_BAD_INPUT      5  /* instance parameters out of range (L, K, d) */
#define FP_STATUS_UNRESOLVED     6  /* |<m>| > 1 at a sample: the truncated operator at this L
                                       is not dissipative for the instance (raise L) */

/* Material of Sec. 2.1 / 2.4.1: saturation magnetisation Ms [A/m], Gilbert
 * damping alpha, gyromagnetic ratio gamma [rad/(s T)], temperature T_B [K]. */
typedef struct {
    double Ms, alpha, gamma, T_B;
} fp_material;

/* Drive field H_DF of Sec. 2 / Sec. 2.4, per lab axis k:
 *     B_k(t) = amp[k] * sin(2 pi freq[k] t + phase[k])     [T]
 * A cosine Lissajous drive has phase pi/2.  One period lasts `period` seconds
 * and is sampled at samples_per_period equidistant times; the output holds
 * output_periods periods after warmup_periods periods:
 *     t_j = (warmup_periods + j / samples_per_period) * period,
 *     j = 0 .. output_periods * samples_per_period - 1.                      */
typedef struct {
    double amp[3];
    double freq[3];
    double phase[3];
    double period;
    int samples_per_period;
    int warmup_periods;
    int output_periods;
    int pad_;
} fp_drive;

/* Integrator controls.  Local error per step (max norm) must stay below
 * atol + rtol * max|c|.  max_steps bounds accepted+rejected steps per
 * instance; newton_max_iter bounds Newton iterations per step;
 * refactor_every bounds how many steps reuse one FP32 factorisation;
 * stages selects the Radau IIA method: 3 (order 5) or 5 (order 9). */
typedef struct {
    double rtol, atol;
    int max_steps;
    int newton_max_iter;
    int refactor_every;
    int checkpoint_every;   /* adjoint checkpoint stride in steps (fp_grad) */
    int stages;
    int pad_;
} fp_tol;

/* One instance (Sec. 2.2 (iii) model m_bar_(D, K, vartheta) at one voxel):
 * offset field h_off = mu0 H_SF(r) [T] in the lab frame, easy axis (theta,
 * phi), anisotropy K [J/m^3], core diameter d [m], truncation degree L
 * (2 <= L <= fp_max_degree()).  64 bytes, 8-byte aligned.                 */
typedef struct {
    double h_off[3];
    double theta, phi;
    double K, d;
    int L;
    int flags;              /* reserved, must be 0 */
} fp_instance;

typedef struct fp_ctx fp_ctx;

/* Largest truncation degree the library supports. */
int fp_max_degree(void);

/* Create a context: copies the material, drive and tolerances, builds the
 * closed-form coupling tables for degrees <= L_max on the current CUDA device.
 * Allocates device memory here and only here.  *out receives the context. */
int fp_setup(const fp_material* mat, const fp_drive* drive, const fp_tol* tol,
             int L_max, fp_ctx** out);

/* Release a context and its device tables.  NULL is accepted. */
int fp_destroy(fp_ctx* ctx);

/* Number of output samples per instance: output_periods * samples_per_period. */
int fp_num_samples(const fp_ctx* ctx);

/* Solve n instances (Sec. 2.1, Eq. FP-general with the readout of
 * Eq. mean_magmom_FP divided by m0).  Layouts (row-major, FP64):
 *   d_inst  [n]            fp_instance, device memory
 *   d_m     [n][S][3]      <m>(t_j) in the lab frame (may be NULL)
 *   d_dmdt  [n][S][3]      d<m>/dt(t_j), exact (l = 1 rows of A(t_j) c) (may be NULL)
 *   d_status[n]            FP_STATUS_* per instance
 *   d_stats [n][4] or NULL accepted steps, rejected steps, Newton iterations,
 *                          factorisations
 * with S = fp_num_samples(ctx).  n == 0 is a no-op.  Instances with a bad L
 * or non-positive K < 0, d <= 0 get FP_STATUS_BAD_INPUT and zero outputs.
 * The launch uses the context's factor scratch and work counter (allocated
 * by fp_setup): calls on one context must not overlap in time (issue them on
 * one stream, or give each stream its own context). */
int fp_solve_batch(fp_ctx* ctx, const fp_instance* d_inst, int n,
                   double* d_m, double* d_dmdt, int* d_status, int* d_stats,
                   void* stream);

/* Normalised signal of Sec. 2.2 (model M1 phi_hat, per unit m0) by the
 * rectangle rule over the LAST output period of d_dmdt:
 *   phi_hat[i][c][k] = (1/S_p) sum_{j<S_p} (p_c . dmdt[i][j0 + j]) e^{-2 pi i j k / S_p}
 * with S_p = samples_per_period, j0 = S - S_p, channel directions p_c
 * (h_channels [C][3], host memory, homogeneous receive coils, Sec. 2.2 (ii)),
 * k = 0..k_max (k_max < S_p).  Output d_phihat [n][C][k_max+1][2] (re, im), FP64. */
int fp_signal(fp_ctx* ctx, const double* d_dmdt, int n, int k_max,
              const double* h_channels, int C, double* d_phihat, void* stream);

/* ---------------------------------------------------------------------------
 * Uneven sweeps: tens of thousands of instances of different truncation degree
 * L and stiffness in one submission (the instances are independent, Sec. 2.1,
 * last paragraph; the parameter sweeps of Sec. 2.4.1).  fp_sweep_plan groups
 * the host copy of the instances into buckets of equal launch degree (L rounded
 * up to a multiple of bucket_width, at most the context's L_max), orders the
 * buckets by decreasing L and each bucket by decreasing estimated cost
 * (sigma + b_T |B|max), and allocates the device order array and work
 * counters (the only allocations; plan before any stream capture).
 * fp_sweep_run solves the instances d_inst (device copy of the same records,
 * same order) into the layouts of fp_solve_batch: one persistent launch per
 * bucket whose CTAs take instances from a work counter, the buckets forked
 * onto side streams and joined; the whole submission is captured into a CUDA
 * graph on the first run and replayed while (d_inst, d_m, d_dmdt, d_status,
 * d_stats, stream) stay the same.  stream must not be the legacy default
 * stream (it cannot be captured).  fp_sweep_autotune times, per bucket, a
 * strided sample of `sample` instances under each candidate (Radau stages 3
 * or 5, refactorisation every 8 or 16 steps) and keeps the fastest candidate
 * whose sample converged; it synchronises the stream and overwrites the
 * sampled instances' outputs.  A plan borrows ctx, which must outlive it.
 * ------------------------------------------------------------------------- */
typedef struct fp_sweep fp_sweep;

int fp_sweep_plan(fp_ctx* ctx, const fp_instance* h_inst, int n, int bucket_width, fp_sweep** out);
/* The host part of fp_sweep_plan, without a context or a GPU: h_order[n]
 * receives the queue order (instance indices, buckets of decreasing launch
 * degree, each by decreasing sigma + b_T |B|max), h_bucket_L / h_bucket_count
 * (at least FP_L_MAX_ANY entries, may be NULL) each bucket's launch degree and
 * size, *n_buckets their number.  Instances with L outside [2, L_max] are
 * FP_EINVAL. */
int fp_sweep_order(const fp_material* mat, const fp_drive* drv, int L_max, const fp_instance* h_inst, int n,
                   int bucket_width, int* h_order, int* h_bucket_L, int* h_bucket_count, int* n_buckets);
/* Host only.  Truncation degree per instance (a reading of the paper, which
 * fixes no degree): L = clamp(L_min, L_max, ceil(2 + 5.5 sqrt(sigma + xi_max))),
 * sigma = K V / (kB T), xi_max = bT (|h_off| + |drive amplitude|), V = pi d^3 / 6,
 * bT = V Ms / (kB T).  The coefficients fit the degree at which the
 * spherical-harmonic tail of the Boltzmann density beyond L - 2 falls below
 * 1e-8 of its mean (sigma in [0.5, 12], xi in [0, 20]).  h_L[n] receives the
 * degrees; sweeps plan with the same rule. */
int fp_truncation_degree(const fp_material* mat, const fp_drive* drv, const fp_instance* h_inst, int n, int L_min,
                         int L_max, int* h_L);
int fp_sweep_run(fp_sweep* sw, const fp_instance* d_inst, double* d_m, double* d_dmdt, int* d_status,
                 int* d_stats, void* stream);
int fp_sweep_autotune(fp_sweep* sw, const fp_instance* d_inst, double* d_m, double* d_dmdt, int* d_status,
                      int sample, void* stream);
/* Buckets of a plan: their count, and per bucket (arrays of at least
 * FP_L_MAX_ANY entries, each may be NULL) launch degree, instance count,
 * stages, refactorisation interval and the autotuned sample time [ms]. */
#define FP_L_MAX_ANY 64
int fp_sweep_info(const fp_sweep* sw, int* n_buckets, int* h_L, int* h_count, int* h_stages, int* h_refactor,
                  float* h_tuned_ms);
int fp_sweep_destroy(fp_sweep* sw);

/* Device workspace (bytes) that fp_grad needs for n instances: per CTA of the
 * persistent launch, the recorded step sequence (fp_tol.max_steps steps), one
 * checkpoint state every 64 steps, one 65-state segment with the stage
 * increments of its 64 steps, plus the readout cotangents of one period.
 * Negative FP_E* on error. */
long long fp_grad_workspace_bytes(const fp_ctx* ctx, int n);

/* Discrete adjoint of the solve + phi_hat map (differentiation of the fixed,
 * recorded step sequence of the Radau integration; Sec. 2.1 equations as in
 * fp_solve_batch, readout of Sec. 2.2).  Given the cotangent
 *   d_dJ_dphihat [n][C][k_max+1][2] = (dJ/dRe phi_hat, dJ/dIm phi_hat)
 * of a real scalar J, writes
 *   d_grad [n][4] = (dJ/dK, dJ/dd, dJ/dtheta, dJ/dphi)
 * per instance (K in J/m^3, d in m, angles in rad).  The forward pass is
 * re-run inside with checkpoints every 64 steps; each 64-step segment is
 * replayed, and every step's transposed collocation system is solved with FP64
 * residuals.  The initial-state term uses central differences of the Boltzmann
 * projection.  h_channels, C, k_max as in fp_signal.  d_status as in
 * fp_solve_batch; d_stats [n][4] or NULL: forward accepted steps, forward
 * rejected steps, the phase that failed (0 none, 1 forward pass, 2 segment
 * replay, 3 transposed stage solve) and the step index where it failed (-1 if
 * none).  Gradients of instances whose status is not FP_STATUS_OK are 0.
 * d_work: device workspace of
 * work_bytes >= fp_grad_workspace_bytes(ctx, n), 16-byte aligned (FP_EINVAL
 * otherwise; cudaMalloc gives 256), owned by the caller, contents undefined on
 * return.  With 5 stages each CTA's share of it opens with that CTA's FP32
 * factors (131 KB at L_max = 16), the rest of the adjoint state sits in shared
 * memory.  Asynchronous on `stream`. */
int fp_grad(fp_ctx* ctx, const fp_instance* d_inst, int n, int k_max,
            const double* h_channels, int C, const double* d_dJ_dphihat,
            double* d_grad, int* d_status, int* d_stats, void* d_work,
            unsigned long long work_bytes, void* stream);

/* The paper has no counterpart: this is a library convenience.
 * fp_grad without a workspace argument, for callers that may not allocate
 * device memory when they call: a host program that gives this library a
 * fixed device-memory footprint and forbids further cudaMalloc (a plugin inside
 * another runtime, a long-running service that must not grow or fragment its
 * memory), or one that cannot size and keep a workspace of its own.  It
 * allocates nothing: the scratch is a static device array of
 * FP_GRAD_NOALLOC_SCRATCH_BYTES compiled into libfp.so, held by every GPU that
 * loads the library until the process exits.  Arguments, outputs, statuses and
 * stats as in fp_grad.  The scratch bounds how many instances run at once
 * (fewer CTAs, each taking several instances in turn), not n; if a single
 * instance needs more than the array (fp_grad_workspace_bytes(ctx, 1) >
 * FP_GRAD_NOALLOC_SCRATCH_BYTES; lower fp_tol.max_steps or L_max) the call
 * returns FP_EINVAL with the sizes in fp_last_error() and launches nothing.
 * The current device must be the context's.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress), so make that first
 * call before any stream capture.  The address is kept for the life of the
 * process: after a reset of the device (cudaDeviceReset, or a primary-context
 * reset by other code) it is stale, so do not call fp_grad_noalloc on a
 * device that has been reset since its first call.  Every call on a device shares the one
 * array and overwrites what the previous call left there (nothing in it needs
 * to start at zero): calls whose launches may overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller. */
#define FP_GRAD_NOALLOC_SCRATCH_BYTES (32ull << 20)
int fp_grad_noalloc(fp_ctx* ctx, const fp_instance* d_inst, int n, int k_max,
                    const double* h_channels, int C, const double* d_dJ_dphihat,
                    double* d_grad, int* d_status, int* d_stats, void* stream);

/* ---------------------------------------------------------------------------
 * Harmonic surrogate: a multilayer perceptron mapping one instance
 * (offset field B_off [T] (3), easy-axis theta, phi [rad], ln K, ln d) to the
 * leading harmonics of its normalised signal phi_hat (Sec. 2.2, model M1),
 * FP_SUR_OUT = 2 channels x 200 complex harmonics k = 1..200, stored
 * [channel][k-1][re, im].  The paper has no surrogate; the Fokker-Planck solve
 * (fp_solve_batch + fp_signal) produces its training data and is the reference for its error.
 * Layers l = 0..4: z_l = W_l x_l + b_l with x_0 the normalised, zero-padded
 * input (64 wide), x_{l+1} = gelu(z_l) (exact erf form) for l < 4 and the
 * output y = z_4 * out_scale + out_shift; gelu(x) = x (1 + erf(x / sqrt 2)) / 2
 * with erf evaluated by Abramowitz & Stegun 7.1.26 (|error| <= 1.5e-7).  BF16 operands, FP32 accumulation on
 * the tensor cores (tcgen05, TMEM accumulators, TMA-fed shared memory).
 * Weight layouts (row-major, bf16): W_l [N_l][K_l] with K = (64, 512, 512,
 * 512, 512), N = (512, 512, 512, 512, 800); columns 7..63 of W_0 must be 0.
 * ------------------------------------------------------------------------- */
#define FP_SUR_IN 7
#define FP_SUR_KIN 64
#define FP_SUR_HIDDEN 512
#define FP_SUR_LAYERS 5
#define FP_SUR_OUT 800

typedef struct {
    const void* W[FP_SUR_LAYERS];     /* bf16 [N_l][K_l] */
    const float* b[FP_SUR_LAYERS];    /* f32 [N_l] */
    const float* in_shift;            /* f32 [7]: x_norm = (x - in_shift) * in_scale */
    const float* in_scale;            /* f32 [7] */
    const float* out_shift;           /* f32 [800] */
    const float* out_scale;           /* f32 [800] */
} fp_surrogate;

/* Training state: the inference view plus what the optimiser keeps. */
typedef struct {
    fp_surrogate net;                 /* net.W are refreshed from Wm by fp_surrogate_adam */
    void* WT[FP_SUR_LAYERS];          /* bf16 [K_l][N_l], transposed copies (backward) */
    float* Wm[FP_SUR_LAYERS];         /* f32 master weights [N_l][K_l] */
    float* bm[FP_SUR_LAYERS];         /* f32 biases (the buffers net.b points to) */
    float* mW[FP_SUR_LAYERS];         /* Adam first / second moments, f32, like Wm */
    float* vW[FP_SUR_LAYERS];
    float* mb[FP_SUR_LAYERS];         /* like bm */
    float* vb[FP_SUR_LAYERS];
} fp_surrogate_train;

/* Device workspace (bytes) for q queries: inference (training = 0), one
 * gradient evaluation (training = 1; q must then be a multiple of 8), or
 * ensemble inference (training = 2, fp_surrogate_infer_ensemble). */
long long fp_surrogate_workspace_bytes(int q, int training);

/* Surrogate inference: d_x [q][7] f32 -> d_y [q][800] f32.  d_err (device
 * int, required) is OR-ed with a nonzero code if a kernel wait timed out
 * (never expected; the outputs are then undefined).  d_work: workspace of
 * fp_surrogate_workspace_bytes(q, 0) bytes, contents undefined on return.
 * Asynchronous. */
int fp_surrogate_infer(const fp_surrogate* net, const float* d_x, int q, float* d_y, void* d_work,
                       unsigned long long work_bytes, int* d_err, void* stream);

/* Two-network ensemble (the paper has no surrogate; its fallback and error
 * judge is the solver): d_mean [q][800] = (y_0 + y_1) / 2 and d_spread [q] =
 * ||y_0 - y_1||_2 / (2 ||mean||_2), the members' disagreement used to send a
 * query to the solver.  The second network's last GEMM folds its output into
 * the mean in its epilogue and accumulates both norms per query there.
 * Workspace fp_surrogate_workspace_bytes(q, 2); otherwise as
 * fp_surrogate_infer. */
int fp_surrogate_infer_ensemble(const fp_surrogate* net0, const fp_surrogate* net1, const float* d_x, int q,
                                float* d_mean, float* d_spread, void* d_work, unsigned long long work_bytes,
                                int* d_err, void* stream);

/* Loss and gradients of one batch: loss = sum over queries and outputs of
 * (z_4 - (y - out_shift)/out_scale)^2, written to *d_loss (f32, overwritten);
 * d_gW[l] f32 [N_l][K_l] and d_gb[l] f32 [N_l] receive the gradients of
 * loss / (q * 800) (mean squared error in normalised output units).  Uses the
 * bf16 weights t->net.W, t->WT and biases.  Asynchronous. */
int fp_surrogate_grad(const fp_surrogate_train* t, const float* d_x, const float* d_y, int q, float* d_loss,
                      float* const* d_gW, float* const* d_gb, void* d_work, unsigned long long work_bytes,
                      int* d_err, void* stream);

/* Adam step (bias-corrected, step >= 1) on the master weights and biases from
 * the gradients, then refresh the bf16 copies t->net.W and t->WT.  step = 0
 * only refreshes the copies (after initialising Wm).  Asynchronous. */
int fp_surrogate_adam(const fp_surrogate_train* t, float* const* d_gW, float* const* d_gb, float lr, float beta1,
                      float beta2, float eps, int step, void* stream);

/* ---------------------------------------------------------------------------
 * Data-driven system-matrix models (Sec. 2.2) and distance measures (Sec. 2.3).
 * System matrices are laid out like fp_signal's output, [voxel][channel][k]
 * complex (re, im), k = 0..K1-1.
 * ------------------------------------------------------------------------- */

/* Model M0 (Sec. 2.2, Eq. Langevin): the equilibrium mean moment
 *     <m>_equ(t) = L(bT |B|) B / |B|,  L(x) = coth x - 1/x,  bT = V Ms / (kB T),
 * V = pi d^3 / 6, B(t) = h_off + drive (the context's drive, schedule and
 * material; K, theta, phi are ignored), and its exact time derivative, at the
 * output samples of fp_solve_batch and in its layouts d_m, d_dmdt [n][S][3]
 * (either may be NULL, not both).  fp_signal on d_dmdt gives M0's phi_hat_D.
 * Instances with d <= 0 or flags != 0 get zero outputs. */
int fp_equilibrium(fp_ctx* ctx, const fp_instance* d_inst, int n, double* d_m, double* d_dmdt, void* stream);

/* Model M1 (and M0) fit of Sec. 2.2 ("Technical details"), for Q dictionary
 * elements Phi_q against one measured system matrix S:
 *     a_q[c][k] = S_k conj(Phi_q,k)^T / ||Phi_q,k||_2^2        (row k, channel c)
 *     eps_q[c][k] = (1/sqrt(N)) ||S_k - a_q[c][k] Phi_q,k||_2 / ||S_k||_inf   (Eq. error1)
 * d_phi [Q][N][C][K1][2], d_S [N][C][K1][2]; outputs d_a [Q][C][K1][2],
 * d_eps [Q][C][K1], d_smax [C][K1] (= ||S_k||_inf).  A row with Phi = 0 gets
 * a = 0; a row with S = 0 gets eps = 0.  Q <= 65535.  Two passes over the data. */
int fp_m1_fit(const double* d_phi, int Q, const double* d_S, int N, int C, int K1, double* d_a, double* d_eps,
              double* d_smax, void* stream);

/* Distance measures of Sec. 2.3 from row errors d_eps [A][C][K1] (A angles,
 * C receive channels): per frequency eps_freq[k] = sqrt(mean_{angle, c}
 * eps^2) into d_eps_freq [K1] (may be NULL), and the global measure
 * (eq. globalMeasure) sqrt(mean_{k in I_freq} eps_freq[k]^2) into
 * *d_eps_global, with the nk rows d_ks (device ints, each < K1). */
int fp_nrmse(const double* d_eps, int A, int C, int K1, const int* d_ks, int nk, double* d_eps_freq,
             double* d_eps_global, void* stream);

/* Model M2, second step (Sec. 2.2, eq. LSfitM2 / eq. LSfitM2_alternative).
 * Dictionary Psi_{theta,j} = diag(a_{theta,j}) Phi_{theta,j} for A angles and
 * J parameter tuples (D, K); rows r = (angle, voxel, channel, k in ks), each
 * weighted by Sigma = 1 / ||S_{theta,k}||_inf per channel (d_smax [A][C][K1]
 * as fp_m1_fit returns it per angle; a zero entry drops the row).  With the
 * columns M[r][j] = Sigma Psi_{theta,j} and y[r] = Sigma S_theta, fp_m2_gram
 * writes the complex Gram matrix of [M | y] into d_G [(J+1)][(J+1)][2]:
 *     G[i][j] = sum_r conj(M[r][i]) M[r][j]   (column J is y)
 * for i <= j (the Hermitian upper triangle; entries below it are left
 * unspecified).  d_phi [A][J][N][C][K1][2], d_a [A][J][C][K1][2],
 * d_S [A][N][C][K1][2], d_ks [nk] rows (device ints < K1).  FP64, summed by
 * row blocks with atomic adds (the summation order varies between calls);
 * d_G is cleared on the stream first; fp_m2_gram_bytes(J) gives its size. */
long long fp_m2_gram_bytes(int J);
int fp_m2_gram(const double* d_phi, const double* d_a, const double* d_S, const double* d_smax, int A, int J, int N,
               int C, int K1, const int* d_ks, int nk, double* d_G, void* stream);

/* Host only.  Non-negative M2 weights from the Gram matrix h_G of fp_m2_gram
 * (host copy; its upper triangle is read).  M^H M = V diag(s^2) V^H gives the truncated problem of
 * eq. approx_low_rank, min_{w >= 0} ||U_s^H (M w - y)||_2^2 with
 * U_s^H M = diag(s_1..s_s) V_s^H and U_s^H y = diag(1/s) V_s^H M^H y, its
 * complex rows split into real and imaginary parts; s = s_rank (<= 0: all
 * numerically nonzero singular values).  The quadratic program
 * min 1/2 w^T Q w + f^T w, w >= 0 is solved by a primal-dual interior-point
 * method; the weight of a column that is zero in the truncated problem (it
 * cannot change the objective) is set to 0, as are all weights at rank 0.
 * Outputs: h_w [J], *h_objective = the truncated objective,
 * *h_residual = ||M w - y||_2^2, h_sv [J] = singular values of M (each of
 * the three may be NULL).  Returns the rank s used (>= 0), or a negative
 * FP_E* code (FP_EUNSUPPORTED if the iteration does not converge).  The
 * eigen-decomposition is a cyclic Jacobi method on a 2J x 2J real matrix:
 * O(J^3) per sweep. */
int fp_m2_solve(const double* h_G, int J, int s_rank, double* h_w, double* h_objective, double* h_residual,
                double* h_sv);

/* Host only.  Mixing orders of frequency index k (Eq. mix):
 * k = m_x n_dens + m_y (n_dens + 1) with the smallest |m_x| + |m_y|; ties go
 * to the smaller |m_x|, then to m_x >= 0. */
int fp_mixing_order(int k, int n_dens, int* mx, int* my);

/* Host only.  I_freq of Sec. 2.3: the distinct k(m_x, m_y) <= k_limit for
 * 0 <= m_x <= M_x, 0 <= m_y <= M_y without the orders (0,0), (0,1), (1,0), in
 * increasing order; the first cap of them into h_ks, their number into *count. */
int fp_freq_index_set(int M_x, int M_y, int n_dens, int k_limit, int* h_ks, int cap, int* count);

/* Diagnostic (host only, no GPU needed): dense Galerkin matrix A of
 * dc/dt = A c (Eq. FP-general tested against the real SH basis) for one
 * instance in the EASY-AXIS frame (n = z), with the field B_nframe [T] already
 * rotated into that frame, built from the same closed-form coupling tables
 * the kernels use.  h_inst->L in [2, 64]; theta/phi are ignored.  h_A
 * receives N*N doubles row-major, A[target][source], N = (L+1)^2, index
 * i = l*l + l + m (real SH without Condon-Shortley phase). */
int fp_operator_dense(const fp_material* mat, const fp_instance* h_inst,
                      const double B_nframe[3], double* h_A);

/* Measurement utility (the paper has no counterpart): FP64 FMA throughput of
 * the current device in GFLOP/s (2 flops per FMA), from 8 independent FMA
 * chains per thread on 8 CTAs per SM.  Allocates and frees 32 KB of device
 * memory; synchronous.  Used as the roofline denominator of the solver. */
int fp_peak_fp64(double* gflops);

/* Text for a status or error code, and the last error message. */
const char* fp_status_str(int code);
const char* fp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FP_H_ */
