/*
 * etd.h -- C ABI of the GB300 (sm_103a) ETD2RK-DS library.
 *
 * The library advances the semi-discrete reaction-diffusion system
 *     u_t + A_h u = f(t, u)   on (0,1)^d, d = 2 or 3, homogeneous Dirichlet,
 * A_h = -kappa Laplace_h + q (Section 2.1: second-order centred differences,
 * n interior points per axis, h = 1/(n+1)), with the Pade-based
 * dimension-split ETD2RK scheme of Section 3.1, eq. (13)-(14) in 2D and
 * eq. (15)-(16) in 3D, by the Sylvester (diagonalisation) route of Section 3.3.2:
 * every shifted 1D solve becomes a product with the eigenvector matrix P of the
 * 1D operator, a Hadamard scaling by precomputed rational-factor grids, and a
 * product with P again (Algorithms 1-2, in matrix-matrix form per Remark 2 of
 * Section 3.4).
 *
 * Conventions shared by every call:
 *   - Field layout: [comp][z][y][x], x fastest, contiguous, no boundary values
 *     (the Dirichlet zeros are implicit; Section 2.1 vectorisation order).
 *     Element type: double for ETD_PREC_FP64 and the FP64-split precisions, float for every
 *     other precision.
 *   - Device pointers must be 16-byte aligned device memory of at least
 *     n_comp * n^d elements; host pointers any host memory of that size.
 *   - The caller owns every field pointer. The plan owns P, the grids, all
 *     workspaces and the carried spectral state; etd_plan_destroy frees them.
 *   - Every call returns an etd_status; none aborts or throws. Kernel-side
 *     errors are reported by the next etd_sync (or etd_step_host, which
 *     synchronises): a bounded device wait that gave up (ETD_ERR_TIMEOUT) and,
 *     when the plan checks its field (etd_options.diag_every > 0), a field
 *     with non-finite values or beyond the bound diag_max_abs (ETD_ERR_DIVERGED).
 *   - Calls on one plan must come from one host thread at a time.
 */
#ifndef ETD_H
#define ETD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct etd_plan etd_plan; /* opaque, library-owned */

typedef enum {
    ETD_OK = 0,
    ETD_ERR_INVALID_ARG = 1, /* bad size, pointer, alignment or option */
    ETD_ERR_OOM = 2,         /* a device allocation failed */
    ETD_ERR_CUDA = 3,        /* a CUDA runtime or driver call failed */
    ETD_ERR_UNSUPPORTED = 4, /* valid request the library or the GPU cannot run */
    ETD_ERR_DIVERGED = 5,    /* non-finite values or |u| beyond diag_max_abs (in-step check, etd_field_stats) */
    ETD_ERR_TIMEOUT = 6      /* a device-side wait exceeded its time limit */
} etd_status;

/* Arithmetic of the eigen-transforms (the dense products with P). */
enum {
    ETD_PREC_FP64 = 0,   /* double fields and state, FP64 CUDA-core products */
    ETD_PREC_FP32 = 1,   /* float fields, FP32 CUDA-core products */
    ETD_PREC_TF32 = 2,   /* float fields, one TF32 tensor-core product */
    ETD_PREC_TF32X3 = 3, /* float fields, split TF32: hi*hi + hi*lo + lo*hi */
    ETD_PREC_BF16X3 = 4, /* float fields, BF16 hi/lo split, three products */
    ETD_PREC_BF16X6 = 5, /* float fields, BF16 hi/mid/lo split, six products in every pass,
                            correction products in their own accumulator (the most accurate
                            mode with float fields: within 1e-6 of FP64 for runs of up to about
                            150 steps of the 2D FitzHugh-Nagumo workload, 4.6e-6 over 1000) */
    ETD_PREC_TF32X6 = 6, /* float fields, TF32 hi/mid/lo split, six products, as BF16X6 */
    ETD_PREC_DST32 = 7,  /* float fields, every transform as fast sine transforms (FFT-based DST-I
                            in FP32 on CUDA cores) instead of the dense product with P: a
                            comparison path, not the paper's dense-eigenbasis method; needs
                            m + 1 a power of two, 16 <= m + 1 <= 8192 */
    ETD_PREC_FP64_SPLIT = 8, /* (default) double fields and state; every product with P in FP64 accuracy on the
                            BF16 tensor cores: each operand row cut into six balanced 8-bit integer
                            slices below a power-of-two scale (P likewise), the 21 slice products of
                            weight >= 2^-40 accumulated exactly, the result formed in FP64 */
    ETD_PREC_FP64_SPLIT40 = 9, /* as ETD_PREC_FP64_SPLIT with five slices (40 bits below each row's
                            scale, 15 slice products): about 2^-40 relative error per product
                            instead of 2^-48, for results held to 1e-6 rather than 1e-10 */
    ETD_PREC_FP64_SPLIT32 = 10 /* four slices (32 bits, 10 slice products): about 2^-32 per product */
};
/* In every split mode (X3, X6) the two transforms whose error stays in the
 * result, U -> U^ when the carried spectral state is (re)built and the
 * transform that returns the field, use three pieces, six products, a separate
 * accumulator for the five correction products and compensated sums.
 * The carried spectral state and the factor grids hold more than FP32
 * precision: FP64 for ETD_PREC_FP64, double-float pairs (hi + lo, about 48
 * bits) for every other precision. */

/* Reaction f(t, u), evaluated pointwise. */
enum {
    ETD_RX_NONE = 0,       /* f = 0 */
    ETD_RX_LINEAR = 1,     /* f = c u; rx_params[0] = c; any n_comp */
    ETD_RX_ALLEN_CAHN = 2, /* f = u - u^3; n_comp = 1 (Example 5.1 without forcing) */
    ETD_RX_FHN = 3,        /* FitzHugh-Nagumo (Example 5.3), n_comp = 2:
                              f_u = u - c3 u^3 - v, f_v = eps (u - a v - b);
                              rx_params = {c3, eps, a, b} */
    ETD_RX_SINGULAR = 4,   /* f = rho u / (1 - u) (Example 5.2); rx_params[0] = rho; n_comp = 1 */
    ETD_RX_AC_FORCED = 5   /* f = u (1 - u^2) + psi(x, t) (Example 5.1): psi makes
                              u = e^{-lambda t} prod sin(pi x_i) exact, with
                              -kappa Lap u0 = d pi^2 kappa u0; rx_params[0] = lambda;
                              n_comp = 1; time-dependent (see etd_set_time) */
};

/* Time-integration factor family, the pade_order argument. */
enum {
    ETD_EXACT_EXP = 0, /* exact exponentials of eq. (9)-(10): e^{-x}, phi_1, phi_2 */
    ETD_PADE_02 = 2,   /* P_{0,2}: Q_1, Q_2, Q_3 of Section 3.1 */
    ETD_PADE_04 = 4    /* P_{0,4}: R_1, R_2, R_3 of Section 5 */
};

typedef struct {
    int precision;         /* ETD_PREC_*, default ETD_PREC_FP64_SPLIT (within 1e-10 of FP64 over whole
                              runs; double fields) */
    int reaction;          /* ETD_RX_*, default ETD_RX_ALLEN_CAHN */
    double rx_params[8];   /* reaction parameters, see ETD_RX_* */
    int n_comp;            /* 1 or 2; default 1 */
    double kappa_comp[2];  /* per-component diffusivity; <= 0 means "use kappa" */
    void* stream;          /* cudaStream_t the plan launches on; NULL = legacy default */
    int flags;             /* ETD_FLAG_* bits, default 0 */
    int diag_every;        /* in-step field check (step a8) every diag_every time steps; 0 (default) = off */
    double diag_max_abs;   /* bound on max |u| for that check; <= 0 (default) = only non-finite values */
} etd_options;

/*
 * In-step field check (diag_every = k > 0). The stability theorem of Section 4
 * bounds max |U^n| by a constant M_* independent of n and tau; a field that
 * leaves such a bound, or holds NaN/Inf, means the run has failed. After every
 * k-th time step of etd_step (counted over the plan's life) the plan reduces
 * max |u| and the number of non-finite values of the returned field in FP64 on
 * the device, with no host synchronisation. When the field has a non-finite
 * value, or max |u| > diag_max_abs > 0, the plan raises its error flag: later
 * tensor-core passes of the plan return at once, and the next etd_sync returns
 * ETD_ERR_DIVERGED (its etd_last_error names the step, max |u| and the count),
 * clears the flag and forgets the carried spectral state. An ensemble
 * (etd_batch_create) checks every group's fields after the last step of each
 * etd_batch_step call.
 */

/*
 * ETD_FLAG_AUTOTUNE: at plan creation (and for each group of an ensemble),
 * time every candidate configuration of the tensor-core pass (one-tile-per-CTA
 * kernel at its tile widths, persistent kernel) on the plan's own buffers, a
 * few launches each with CUDA events on the plan stream, and keep the fastest.
 * Choices are cached per (grid, batch, precision) within the process, so later
 * plans of the same shape reuse them. Without the flag a fixed rule chooses.
 * Plan creation then launches kernels and synchronises its stream.
 */
#define ETD_FLAG_AUTOTUNE 1

/* Performance-relevant facts of a plan (for benchmarks and roofline figures). */
typedef struct {
    int d, n, n_comp, precision;
    int products;                /* tensor-core products per MMA tile (1, 3, 6, or 21 / 15 / 10 slice products for
                                    ETD_PREC_FP64_SPLIT / _SPLIT40 / _SPLIT32; 0 for CUDA cores) */
    int gemms_per_step;          /* transform passes per time step (8 in 2D, 12 in 3D) */
    long long unknowns;          /* n_comp * n^d */
    double gemm_flops;           /* algorithmic flops of one pass, all components: 2 n^(d+1) n_comp */
    double step_flops;           /* algorithmic flops of one time step (16 n or 24 n per unknown) */
    long long workspace_bytes;   /* device memory the plan holds */
    int pass_persistent[2];      /* tensor-core pass configuration of the per-step passes [0] and of
                                    the state-building / returned-field transforms [1]: 1 = the
                                    persistent kernel, 0 = one tile per CTA */
    int pass_tile_n[2];          /* tile width (columns) of those configurations; 0 without tensor cores */
    double step_bytes;           /* algorithmic DRAM bytes of one time step's transform passes: every operand
                                    piece, basis piece, spectral state value and output field value read or
                                    written once per pass (reaction kernels not included) */
    int kernels_per_pass;        /* kernel launches of one transform pass: 1, or 2 (ETD_PREC_DST32: row FFTs
                                    and the transposing epilogue; ETD_PREC_FP64_SPLIT: slices, products) */
} etd_plan_info;

/* Fill *opt with the defaults listed above. */
etd_status etd_options_default(etd_options* opt);

/*
 * Create a plan for one problem (Section 2.1 operator, Section 3.1 scheme).
 *   d          2 or 3
 *   m          interior points per axis (n), 2 <= m <= 16384 (2D), 2 <= m <= 1024 (3D)
 *   kappa      diffusivity > 0 (component 0 unless kappa_comp overrides)
 *   q          potential >= 0, split q/d per axis
 *   dt         time step tau > 0
 *   pade_order ETD_PADE_02, ETD_PADE_04 or ETD_EXACT_EXP
 *   opt        NULL for defaults
 * Precomputes (FP64 on the host) the eigenvectors P (closed-form sine basis)
 * and the factor grids E_l(tau lambda_k), allocates every workspace, and
 * returns the plan in *out (NULL on error).
 */
etd_status etd_plan_create(etd_plan** out, int d, int m, double kappa, double q, double dt, int pade_order,
                           const etd_options* opt);

/*
 * Advance u_dev (device, layout above) in place by n_steps time steps
 * (eq. (13)-(16)); the plan's time advances by n_steps * dt. Asynchronous on
 * the plan stream. The plan carries the spectral coefficients of u between
 * calls; call etd_plan_invalidate after writing u_dev yourself, or pass a
 * different pointer (the plan then re-derives them).
 */
etd_status etd_step(etd_plan* p, void* u_dev, int n_steps);

/*
 * Same as etd_step for a HOST array u_host: copies it to a plan-owned device
 * field, advances n_steps, copies the result back and synchronises. Page-locked
 * host memory gives asynchronous copies; pageable memory works but is slower.
 * When u_host holds exactly (bit for bit) the field the previous call returned,
 * as in a host-side time-stepping loop, the carried spectral state is kept (a
 * device-side comparison of the copied field decides); any other content
 * rebuilds it, as etd_step does for a new field. The step starts from the field
 * the previous call returned while the copy and the comparison run beside it; a
 * changed field discards that step and is stepped from a rebuilt state (same
 * result, the time of two steps). The result is copied back in four parts on
 * the plan stream and three plan-owned streams (created on the first call, with
 * the plan's other host-step buffers); all four have completed when the call returns.
 */
etd_status etd_step_host(etd_plan* p, void* u_host, int n_steps);

/*
 * Spectral transform of one field (step a2 alone): out = T(in) per component,
 * T(X) = P_x^T X P_y in 2D and the three mode products in 3D. in and out are
 * device fields in the layout above ([comp][l][k] / [comp][p][l][k] for the
 * spectral side). T is its own inverse because P is symmetric and orthogonal.
 */
etd_status etd_transform(etd_plan* p, const void* in_dev, void* out_dev);

/*
 * Ensemble of independent problems stepped together (the batched workload of
 * many instances with uneven grids): instance i has d[i], m[i] interior points,
 * diffusivity kappa[i] (component 1, if any, uses opt->kappa_comp[1] when > 0),
 * potential q[i] and time step dt[i]; pade_order and opt (reaction, precision,
 * n_comp, stream) are shared. Instances on the same grid form one group that
 * shares P and runs as one batched sequence of passes on a stream of its own;
 * groups run concurrently. Time-dependent reactions are rejected. The handle is
 * an etd_plan usable with etd_batch_step, etd_sync, etd_plan_invalidate,
 * etd_get_plan_info, the timing calls and etd_plan_destroy.
 */
etd_status etd_batch_create(etd_plan** out, int count, const int* d, const int* m, const double* kappa,
                            const double* q, const double* dt, int pade_order, const etd_options* opt);

/*
 * Advance every instance by n_steps of its own dt. u_dev[i] is instance i's
 * device field (layout above, 16-byte aligned). Fields are gathered into each
 * group's contiguous buffer, stepped, and scattered back, asynchronously with
 * respect to the plan stream (it waits for every group at the end). Passing the
 * same pointers again resumes the carried spectral states.
 */
etd_status etd_batch_step(etd_plan* p, void* const* u_dev, int n_steps);

/*
 * Adjoint (reverse-mode derivative) of n_steps time steps of a single plan.
 * The forward window starts from u_ckpt (device field, the state at its first
 * step). On entry lambda_dev holds dL/dU at the end of the window; on exit it
 * holds dL/dU at u_ckpt. dL/dkappa_c (c < n_comp) is ADDED to grad_kappa[c] and
 * dL/d rx_params[i] (i < 4; FitzHugh-Nagumo: c3, eps, a, b; linear: c;
 * singular: rho) to grad_rx[i]; either pointer may be NULL. The window's
 * forward states are recomputed on the device (memory: n_steps fields).
 * Per step (S = E_1(tau A_2), X_l = E_l(tau A_1), all symmetric and commuting):
 *   Gbar = tau X3 Ubar+, Wbar = Ubar+ + J_f(W)^T Gbar,
 *   Fbar = tau X2 S Wbar - S Gbar, Ubar = X1 S Wbar + J_f(U)^T Fbar.
 * Synchronises. Autonomous reactions only (ETD_RX_AC_FORCED: UNSUPPORTED).
 */
etd_status etd_step_adjoint(etd_plan* p, const void* u_ckpt, void* lambda_dev, int n_steps, double* grad_kappa,
                            double* grad_rx);

/*
 * Failure-path self test (no counterpart in the paper): launches, on the plan
 * stream, a one-CTA kernel whose bounded device wait (the same routine the
 * transform kernels use, limit limit_ms in (0, 1000]) has nothing to wait for,
 * so it runs out, raises the plan's timeout flag and returns. The next etd_sync
 * then returns ETD_ERR_TIMEOUT and clears the flag; the plan stays usable.
 */
etd_status etd_selftest_wait_timeout(etd_plan* p, double limit_ms);

/* Forget the carried spectral state (after the caller changed u_dev). */
etd_status etd_plan_invalidate(etd_plan* p);

/* Set the plan time t (used by time-dependent reactions; default 0). */
etd_status etd_set_time(etd_plan* p, double t);

/* Wait for the plan stream; report device-side errors raised since the last sync. */
etd_status etd_sync(etd_plan* p);

/*
 * FP64 diagnostics of a device field (step a8, on demand): *max_abs = max |u| and
 * *n_nonfinite = number of NaN/Inf entries over all components. Synchronises.
 * Returns ETD_ERR_DIVERGED when n_nonfinite > 0 (outputs still written).
 */
etd_status etd_field_stats(etd_plan* p, const void* u_dev, double* max_abs, long long* n_nonfinite);

/* Copy the plan's facts into *info. */
etd_status etd_get_plan_info(const etd_plan* p, etd_plan_info* info);

/*
 * Kernel timing: when enabled, every launch of the plan is bracketed by CUDA
 * events on the plan stream. etd_kernel_times (after etd_sync) returns, for
 * kind 0 = transform passes of the time steps, 1 = pointwise reaction/split
 * kernels, 2 = the accurate transform passes (state rebuild and returned field,
 * the split modes only), the summed milliseconds and launch count since the
 * last call for that kind.
 */
etd_status etd_set_timing(etd_plan* p, int enable);
etd_status etd_kernel_times(etd_plan* p, int kind, double* total_ms, long long* launches);

/*
 * Spectral transform without device allocation. The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory at
 * the time of the call (a host framework's caching allocator has reserved the
 * GPU's memory, or a latency-critical loop cannot afford the device-wide
 * synchronisation of cudaFree).
 *   out_dev = T(in_dev) per component, the transform of etd_transform with FP32
 *   CUDA-core products; fields float32, [comp][z][y][x], device memory, caller-owned.
 *   d 2 or 3, n >= 2, n_comp 1 or 2, stream a cudaStream_t (NULL = legacy default).
 * Workspace: a static device array of ETD_NOALLOC_MAX_ELEMS floats (16 MiB)
 * that every GPU loading the library holds until the process exits; a call needs
 * n^2 + k n_comp n^d floats (k = 1 in 2D, 2 in 3D) and returns ETD_ERR_INVALID_ARG
 * beyond that. The call allocates nothing. Its first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture. The address is kept per device
 * together with the CUDA context's id; after cudaDeviceReset (a new context, the
 * array loaded again) the next call repeats the look-up, so make it outside a
 * capture as well. All calls share the array and it keeps the last call's
 * contents: calls that overlap on the GPU (other streams, other host threads)
 * race. Launch failures are read from each launch's own return code; an error
 * that earlier work left pending is not cleared. Asynchronous on `stream`.
 */
#define ETD_NOALLOC_MAX_ELEMS 4194304
etd_status etd_transform_noalloc(int d, int n, int n_comp, const void* in_dev, void* out_dev, void* stream);

/* Release every resource of the plan. NULL-safe. */
etd_status etd_plan_destroy(etd_plan* p);

/* Static description of a status code. */
const char* etd_status_string(etd_status s);

/* Message of the last failing call on this host thread ("" if none). */
const char* etd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ETD_H */
