/*
 * floquet.h - C ABI of the GB300 (sm_103a) Magnus-Chebyshev Floquet propagator.
 *
 * Method (arXiv:1508.07621): the Floquet operator U_T of H(t) = H0 + f(t) H1 (Eq. 13) is
 * built by propagating the N x N identity over one period T (§3, last paragraph) through a
 * chain of M single-step propagators (Eq. 9).  Each step uses the 4th-order midpoint Magnus
 * exponent Omega_m = a_m H0 + b_m H1 + c_m i[H0,H1] (Eq. 14 truncated after its leading
 * commutator; a_m = h, b_m = h f + h^3 f''/24, c_m = h^3 f'/12 at the step midpoint), shifted
 * and rescaled to spectrum [-1, 1] (Eq. 11), and applies exp(-i Omega_m) by the Chebyshev
 * recurrence (Eq. 10) with Bessel weights a_0 = J_0(R), a_l = 2 J_l(R), R = h Delta E (Eq. 12).
 * hbar = 1 throughout.
 *
 * Stages of the path, as the sources label them
 *  a1  host planning: Magnus scalars per step, spectral bounds, R, L, Bessel weights
 *  a2  the rescaled step exponent Omega~_m (Eq. 11), formed in FP64 once per step
 *  a3  one dense Chebyshev term (a complex N x N product, Eq. 10)
 *  a4  one tridiagonal Chebyshev term
 *  a5  the Bessel-weighted accumulation, fused into the term's epilogue
 *  a6  the step close (phase e^{-i beta h}) and the chaining of the M steps
 *  a7  the unitarity defect of U_T
 *  a8  operand preparation for the tensor cores (BF16 or fixed-point slices)
 *  a9  many plans' U_T builds in one CUDA graph
 *  a10 the adjoint chain and the gradient of the gate-fidelity loss in the drive amplitudes
 *
 * Conventions
 *  - Complex numbers at the boundary are interleaved (re, im) doubles, i.e. C99 double
 *    complex / torch.complex128.
 *  - A "state block" of ncols states is ncols x N, row-major: row r is state r, a contiguous
 *    length-N vector (the paper stores its initial vectors as rows, §5).
 *  - U_T is returned as the N x N row-major matrix U[i][j] = <i|U_T|j>: column j is basis
 *    vector j propagated over the period.
 *  - U_T = U_M ... U_1 (the earliest step acts first on column states).
 *
 * Ownership and memory
 *  - Every device pointer argument is allocated and owned by the caller.  The library never
 *    frees caller memory.  Device memory the library allocates itself is limited to what
 *    floquet_plan_create makes (operators, per-step scalars, a status word); it is released
 *    by floquet_plan_destroy.  All scratch space is the caller's workspace, whose size is
 *    given by floquet_workspace_size / floquet_grad_workspace_size.
 *  - Host arrays passed to floquet_plan_create are copied; the caller keeps ownership.
 *
 * Streams and errors
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Compute
 *    calls only enqueue work on it and return without synchronising, except where stated.
 *  - Every call returns an fq_status.  Argument errors are reported before any work is
 *    enqueued.  Device-side checks (a propagated entry larger than the bound implied by
 *    unitarity, a Clenshaw vector above its bound, a state whose norm drifts by more than
 *    1e-3 relative over the chain, or NaN) set bits in a per-plan status word; floquet_check_status
 *    synchronises the stream, returns FQ_EBOUND if any bit was set, and clears it.  The
 *    library never traps or aborts.  floquet_last_error returns a message for the last
 *    failing call of the calling thread.
 *  - Problems are checked in host planning: every operator entry, drive parameter, drive sample
 *    and caller bound must be finite (else FQ_EINVAL), and R = h Delta E must be at most 16384
 *    (about R + 300 Chebyshev products per step; beyond it FQ_EUNSUPPORTED: use more steps).
 *  - No C++ exception leaves the library: a failed host allocation is FQ_ENOMEM.
 *  - Plans are not thread-safe: one plan must not be used by two concurrent calls.
 */
#ifndef FLOQUET_H
#define FLOQUET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fq_status {
  FQ_OK = 0,
  FQ_EINVAL = 1,        /* invalid argument (NULL pointer, bad size, workspace too small) */
  FQ_ENOMEM = 2,        /* device or host allocation failed in floquet_plan_create */
  FQ_ECUDA = 3,         /* a CUDA runtime call failed; see floquet_last_error */
  FQ_EBOUND = 4,        /* device check: |entry| above the unitarity bound, or NaN */
  FQ_ETIMEOUT = 5,      /* a bounded device wait gave up */
  FQ_EUNSUPPORTED = 6   /* valid request the library does not implement */
} fq_status;

typedef enum fq_format {
  FQ_DENSE = 0,         /* H0, H1 dense real-symmetric N x N, row-major */
  FQ_TRIDIAG = 1        /* H0 real-symmetric tridiagonal, H1 real diagonal */
} fq_format;

typedef enum fq_precision {
  FQ_FP64 = 0,          /* every product and accumulation in FP64 (baseline path) */
  FQ_FP32 = 1,          /* FP32 storage and FP32 arithmetic (tridiagonal format) */
  FQ_BF16X3 = 2,        /* dense: 2-slice BF16 split, products hi*hi + hi*lo + lo*hi, FP32 accumulate */
  FQ_BF16X6 = 3,        /* dense: 3-slice BF16 split, 6 slice products, FP32 accumulate */
  FQ_DF32 = 4,          /* double-float arithmetic (each value a pair of FP32 numbers, about 48
                           significant bits) on the FP32 pipes; FP64 states in HBM; FP64-level
                           results.  Tridiagonal: tiled kernel (L <= 128); dense: resident
                           kernel (N <= 128, L <= 128); FQ_EUNSUPPORTED otherwise */
  FQ_OZAKI = 5          /* FP64 emulation on the BF16 tensor cores (Ozaki-style splitting): six
                           8-bit fixed-point slices per row, 21 slice products, exact FP32 partial
                           sums combined in double-float; FP64-level results.  Dense: per
                           Chebyshev term, FP64 states.  Tridiagonal: the band kernel
                           (FQ_KERNEL_BAND, L <= 47), double-float states */
} fq_precision;

typedef enum fq_drive_kind {
  FQ_DRIVE_COS = 0,       /* f(t) = f_dc + f_ac cos(omega t + phi0) */
  FQ_DRIVE_PIECEWISE = 1  /* f constant on each step; values given per call (floquet_grad) */
} fq_drive_kind;

typedef enum fq_kernel {
  FQ_KERNEL_AUTO = 0,       /* resident kernel when it applies, else tiled, else streaming */
  FQ_KERNEL_STREAM = 1,     /* tridiagonal: one launch per Chebyshev term, states in HBM;
                               dense FP64: one tiled GEMM launch per term (also for TILED) */
  FQ_KERNEL_RESIDENT = 2,   /* tridiagonal FP32: one CTA per state runs the whole chain on chip
                               (N <= 10240, L <= 128); dense FP64: a cluster of ceil(N/32) CTAs
                               per state runs 64 steps per launch on chip (N <= 128, L <= 128);
                               FQ_EUNSUPPORTED otherwise */
  FQ_KERNEL_TILED = 3,      /* tridiagonal FP64 or FP32, any N, L <= 128: one launch per step, each
                               CTA runs the step's L products on a segment of one state plus L
                               halo rows a side; FQ_EUNSUPPORTED otherwise.  AUTO picks RESIDENT,
                               then TILED, then STREAM. */
  FQ_KERNEL_BAND = 4        /* tridiagonal FQ_OZAKI (the only kernel for it; AUTO selects it),
                               L <= 47: per step the band matrix P_m = e^{-i beta h} sum_k c_k
                               T_k(Omega~_m) of Eqs. 10-12 (2L+1 diagonals) is formed once, and every
                               state is multiplied by it on the tensor cores in FP64 emulation
                               (fixed-point BF16 slices, exact FP32 sums), one windowed product per
                               step; states are double-float pairs between steps */
} fq_kernel;

/* Problem statement (Eq. 13, §3): everything floquet_plan_create needs. */
typedef struct fq_problem {
  int32_t n;                /* Hilbert-space dimension N >= 1 */
  int32_t format;           /* fq_format */
  const double* h0;         /* DENSE: N*N row-major symmetric; TRIDIAG: diagonal, N values */
  const double* h0_off;     /* TRIDIAG: H0[i+1][i] = H0[i][i+1], N-1 values; DENSE: ignored */
  const double* h1;         /* DENSE: N*N row-major symmetric; TRIDIAG: diagonal, N values */
  double period;            /* T > 0 */
  int32_t steps;            /* M >= 1; h = T/M */
  int32_t drive_kind;       /* fq_drive_kind */
  double f_dc, f_ac, omega, phi0;   /* FQ_DRIVE_COS parameters */
  const double* f_steps;    /* FQ_DRIVE_PIECEWISE: M amplitudes used to freeze the spectral
                               bounds (range widened by 10%); later calls pass their own f_m */
  double cheb_tol;          /* truncation |J_{L+1}(R)| < tol; <= 0 selects 1e-14 */
  double e_min, e_max;      /* if e_max > e_min: caller's bounds of Omega/h, used as given */
  int32_t precision;        /* fq_precision */
  int32_t checkpoint_stride;/* floquet_grad: X_m stored every s steps; <= 0 selects 16 */
  int32_t kernel;           /* fq_kernel: which kernel family runs the chain (tridiagonal, and
                               dense FP64); ignored by the split precisions */
  int32_t tile_n;           /* split path: tensor-core output tile width 64 or 128; 0 = 128 until
                               floquet_autotune picks one */
  int32_t magnus_order;     /* 4 (default, also 0) or 6: Eq. 14 in full with its alphas taken as
                               3-point Gauss-Legendre moments (nine commutators of H0, H1 computed
                               once: on the device for FQ_DENSE, on the host as bands for
                               FQ_TRIDIAG); 6 needs FQ_DRIVE_COS, and a tridiagonal plan FQ_FP64
                               (its Omega~ is heptadiagonal: a streaming FP64 kernel applies it) */
  int32_t cheb_terms;       /* > 0: a fixed number L of Chebyshev products per step (the paper's
                               timing runs use L = 50, Table 1), overriding cheb_tol; at most
                               1024 and at least the R-dependent minimum (L > R); 0: from cheb_tol */
  int32_t tile_k;           /* split path, FQ_BF16X3 with 64-wide tiles: K elements a pipeline
                               stage loads, 32 (four stages) or 64 (two); 0 = 64 until
                               floquet_autotune picks one; other tiles take 32 */
} fq_problem;

typedef struct fq_plan fq_plan;

/* Host-computed planning results (stage a1): bounds (Eq. 11), R and L (Eq. 12). */
typedef struct fq_plan_info {
  int32_t n, steps, L, precision, format, drive_kind;
  double h, e_min, e_max, beta, delta_e, R;
} fq_plan_info;

/* Host planning + upload (§3: Magnus scalars, [H0,H1] computed once, bounds, Bessel
 * coefficients; the set-up part of Algorithm 1).  Uses the current CUDA device; allocates the plan's
 * device copies, which the plan owns until floquet_plan_destroy.  Synchronous.  On failure *plan is
 * NULL and nothing stays allocated: FQ_EINVAL (invalid problem, see fq_problem), FQ_EUNSUPPORTED
 * (a valid combination no kernel implements), FQ_ENOMEM (an allocation failed) or FQ_ECUDA. */
fq_status floquet_plan_create(fq_plan** plan, const fq_problem* problem);

/* Frees the plan and its device memory (synchronises the device first).  NULL is a no-op. */
void floquet_plan_destroy(fq_plan* plan);

/* Copies the plan's planning results (sizes, bounds, R, L) into the caller's *info.  Host only;
 * FQ_EINVAL if either pointer is NULL. */
fq_status floquet_plan_get_info(const fq_plan* plan, fq_plan_info* info);

/* Host planning only (no device needed): fills *info as floquet_plan_create would and writes
 * the Bessel weights a_0 .. a_L (Eq. 12) into coeffs[0 .. min(L, cap-1)] if coeffs is not NULL. */
fq_status floquet_plan_inspect(const fq_problem* problem, fq_plan_info* info, double* coeffs,
                               int32_t cap);

/* Bytes of workspace floquet_propagate / floquet_build_UT need for ncols states (0 for a NULL plan
 * or ncols < 0).  Host only. */
size_t floquet_workspace_size(const fq_plan* plan, int32_t ncols);

/* U_T (the propagation part of Algorithm 1): propagates the N x N identity over all M steps and writes
 * d_U = N x N complex128, U[i][j] = <i|U_T|j> (caller-owned device memory).  d_ws: caller-owned,
 * floquet_workspace_size(plan, N) bytes, 256-byte aligned, else FQ_EINVAL before any work.
 * Asynchronous on `stream`: FQ_ECUDA reports a failed launch; the numerical device checks are read
 * by floquet_check_status. */
fq_status floquet_build_UT(fq_plan* plan, void* d_U, void* d_ws, size_t ws_bytes, void* stream);

/* What a build reports (§8(b)): the planning results it ran with (L, R, the bounds of Eq. 11),
 * the unitarity defect of the U_T it wrote (max |U^+U - 1| entry and Frobenius / sqrt(k) over k
 * evenly spaced columns, FP64 on the device, as floquet_unitarity_defect) and the device time of
 * the build measured by CUDA events on the stream. */
typedef struct fq_report {
  int32_t L, defect_columns;
  double R, e_min, e_max, beta, delta_e;
  double defect_max, defect_fro;
  double build_ms;
} fq_report;

/* floquet_build_UT followed by its report: the same build (same kernels, same result), then the
 * defect over defect_columns evenly spaced columns (1 <= defect_columns <= N; the workspace,
 * free after the build, holds the defect's scratch) and the timing.  Synchronises `stream`.
 * d_ws: floquet_workspace_size(plan, N) bytes, and at least floquet_defect_workspace_size(N) +
 * 4 defect_columns + 256 bytes.  FQ_EINVAL for a NULL report or a bad column count, otherwise as
 * floquet_build_UT; FQ_EBOUND if the build's device checks fired (the report is still filled). */
fq_status floquet_build_UT_report(fq_plan* plan, void* d_U, void* d_ws, size_t ws_bytes, void* stream,
                                  int32_t defect_columns, fq_report* report);

/* Kernel timing, a measurement aid (the paper has no counterpart).  While enabled, the calls that
 * run the tridiagonal chain's step kernel with this plan record a pair of CUDA events on the
 * caller's stream around each launch of that kernel: the band product k_oz_band (FQ_OZAKI), the
 * resident chain k_tri_resident (FQ_FP32, one launch per call) or the double-float step
 * k_tri_tile_dfl (FQ_DF32); other paths record nothing, and nothing is recorded on a stream that
 * is capturing a graph.  floquet_kernel_timing switches this on (enable != 0) or off and clears the
 * record.  floquet_kernel_time waits for the last recorded event and returns the launches recorded
 * since the last read, the sum of their durations in milliseconds and the kernel's name
 * (NUL-terminated, at most name_len - 1 characters; name may be NULL), then clears the record.
 * FQ_EINVAL for a NULL plan or output; FQ_ECUDA if an event could not be created or recorded (the
 * record is cleared).  Calls on one plan must not overlap in time. */
fq_status floquet_kernel_timing(fq_plan* plan, int32_t enable);
fq_status floquet_kernel_time(fq_plan* plan, int32_t* launches, double* total_ms, char* name, int32_t name_len);

/* Propagates a block of ncols states through steps m_begin .. m_end-1 (0-based), i.e.
 * X = U_{m_end} ... U_{m_begin+1} X0 (Eq. 9 restricted to those steps).  d_X0, d_X: ncols x N
 * complex128, row r = state r, caller-owned device memory; d_X may equal d_X0.  FQ_EINVAL for a
 * NULL pointer, ncols < 0 or a range outside 0 <= m_begin <= m_end <= M; m_begin = m_end copies.
 * d_ws as for floquet_build_UT with ncols states.  Asynchronous on `stream`.  Used for the second
 * propagation round of §3 (eigenvectors as initial states) and for resuming a chain. */
fq_status floquet_propagate(fq_plan* plan, const void* d_X0, void* d_X, int32_t ncols,
                            int32_t m_begin, int32_t m_end, void* d_ws, size_t ws_bytes,
                            void* stream);

/* Columns j0 .. j0+ncols-1 of U_T: the basis states e_j of those columns of the identity
 * propagated over all M steps, which is one node's share in the column split of §5 (Fig. 2, the
 * distribute part of Algorithm 1; the columns are independent, so no exchange happens while
 * they propagate).  d_X: ncols x N complex128, caller-owned device memory, row r = column
 * j0 + r of U_T (X[r][i] = <i|U_T|j0+r>), so the blocks of consecutive column ranges concatenate
 * into U_T in column-major order.  d_ws: floquet_columns_workspace_size(plan, ncols) bytes,
 * 256-byte aligned.  FQ_EINVAL for a NULL pointer, ncols < 1 or columns outside [0, N), or a short
 * or misaligned workspace, before any work.  Asynchronous on `stream`. */
size_t floquet_columns_workspace_size(const fq_plan* plan, int32_t ncols);
fq_status floquet_build_UT_columns(fq_plan* plan, int32_t j0, int32_t ncols, void* d_X, void* d_ws,
                                   size_t ws_bytes, void* stream);

/* Unitarity defect (§2: truncated Omega is Hermitian, so every step is unitary):
 * over the k columns listed in d_cols (int32, device; NULL = all N columns, k ignored) of the
 * N x N complex128 d_U, computes max_{c in cols, j} |(U^+ U - 1)[c][j]| and the Frobenius
 * norm of those rows / sqrt(k).  Synchronises `stream`; results in host doubles.
 * d_ws: floquet_defect_workspace_size(n) bytes. */
size_t floquet_defect_workspace_size(int32_t n);
fq_status floquet_unitarity_defect(const void* d_U, int32_t n, const int32_t* d_cols, int32_t k,
                                   void* d_ws, size_t ws_bytes, void* stream,
                                   double* max_abs, double* fro);

/* Gate-fidelity loss and gradient for piecewise-constant drives (plan made with
 * FQ_DRIVE_PIECEWISE, FQ_DENSE): L = 1 - |Tr(W^+ U_T)|^2 / N^2 with W = d_W (N x N complex128,
 * row-major) and U_T built from the amplitudes d_f (M doubles, device); writes *d_loss
 * (1 double, device) and d_grad[m] = dL/df_m (M doubles, device).  Reverse-mode through the
 * Magnus-Chebyshev chain (Clenshaw-form adjoint of Eqs. 10-12) with X_m kept every
 * checkpoint_stride steps and recomputed in between.  Precision FQ_FP64 (SIMT FP64) or
 * FQ_BF16X3 / FQ_BF16X6 (tensor-core products on BF16 slices, FP32 accumulation and FP32
 * state masters; the loss, tau and the gradient sums stay FP64), or FQ_OZAKI (tensor-core FP64
 * emulation, FP64 states and epilogues).  FQ_EUNSUPPORTED otherwise.
 * d_ws: floquet_grad_workspace_size (256-byte aligned), else FQ_EINVAL. */
size_t floquet_grad_workspace_size(const fq_plan* plan);
fq_status floquet_grad(fq_plan* plan, const double* d_f, const void* d_W, double* d_loss,
                       double* d_grad, void* d_ws, size_t ws_bytes, void* stream);

/* Second propagation round (§3, last paragraph): propagates the ncols states d_X0 (ncols x N
 * complex128, row r = state r, e.g. Floquet states from the eigenvectors of U_T) over the period
 * and writes d_avg[r] = <A>_T = (1/T) int_0^T <psi_r(t)|A(t)|psi_r(t)> dt (Eq. 17) for
 * A(t) = a0 H0 + (a1 + s_drive f(t)) H1 (A = H(t): a0 = 1, a1 = 0, s_drive = 1), the integral by
 * composite Simpson over the step boundaries (trapezoid if M is odd).  Cosine-drive plans; dense
 * N <= 8192 (else FQ_EUNSUPPORTED).  d_X0 is not modified; d_avg: ncols device doubles.  All
 * buffers are caller-owned; d_ws: floquet_observable_workspace_size(plan, ncols) bytes, else
 * FQ_EINVAL.  Asynchronous on `stream`. */
size_t floquet_observable_workspace_size(const fq_plan* plan, int32_t ncols);
fq_status floquet_average_observable(fq_plan* plan, const void* d_X0, int32_t ncols, double a0, double a1,
                                     double s_drive, double* d_avg, void* d_ws, size_t ws_bytes, void* stream);

/* Overlap phase error of Eq. 20 (§7) under the reading that fixes its phases: for the ncols
 * Floquet states phi~_r (d_states, ncols x N complex128 rows, unit norm; e.g. those of the U_T of
 * the same drive at step h/2) with quasienergies eps~_r (d_eps, ncols device doubles),
 *   d_sigma[r] = |1 - e^{i eps~_r T} <phi~_r| U_T |phi~_r>|,
 * where U_T phi~_r is the plan's whole chain (step h) applied to the state on the device and the
 * overlap is reduced in FP64.  It is the one-period error of the plan's chain against the exact
 * evolution e^{-i eps~ T} phi~ of the finer Floquet state.  d_states is not modified; every
 * buffer is caller-owned; d_ws: floquet_overlap_workspace_size(plan, ncols) bytes, 256-byte
 * aligned, else FQ_EINVAL.  Asynchronous on `stream`. */
size_t floquet_overlap_workspace_size(const fq_plan* plan, int32_t ncols);
fq_status floquet_overlap_phase_error(fq_plan* plan, const void* d_states, int32_t ncols, const double* d_eps,
                                      double* d_sigma, void* d_ws, size_t ws_bytes, void* stream);

/* Size of the library's static device scratch array used by floquet_build_UT_static. */
#define FLOQUET_STATIC_SCRATCH_BYTES (16u << 20)

/* U_T without any device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc (code embedded in a runtime that owns all device
 * memory, or that must not grow its device footprint after start-up).  It runs the same
 * resident FP32 tridiagonal chain as floquet_build_UT, but takes the problem directly (host
 * arrays, no plan) and keeps every intermediate - operators, per-step scalars, the per-step
 * operator coefficients and frame rotations, and the status word - in one static __device__
 * array of FLOQUET_STATIC_SCRATCH_BYTES that each GPU running it holds until exit.
 *  - Limit: (2M + 1) * rows * 8 bytes plus about 3M * 8 + 4N * 8 bytes must fit in
 *    FLOQUET_STATIC_SCRATCH_BYTES, where rows is the resident kernel's padded row count:
 *    512 for N <= 512, 1024 for N <= 1024, 512 * (ceil(N / 512) rounded up to even) for
 *    N <= 9216, 10240 above
 *    (e.g. N = 701, M = 300 fits; N = 1100 needs 2048 rows, so M <= 511).  Larger needs are
 *    rejected with FQ_EINVAL before any work.
 *  - problem: FQ_TRIDIAG with FQ_FP32, kernel FQ_KERNEL_AUTO or FQ_KERNEL_RESIDENT only
 *    (N <= 10240, L <= 128); anything else returns FQ_EUNSUPPORTED.
 *  - d_U: caller-owned N x N complex128 output, U[i][j] = <i|U_T|j>, as floquet_build_UT.
 *  - Calls no cudaMalloc/cudaFree.  The first call on a device looks up the array's device
 *    address with that device current (make it before any stream capture).  Under CUDA's lazy
 *    module loading (the default) the array is committed on a device at that first call, not
 *    when the library is opened: make the first call at start-up, or set
 *    CUDA_MODULE_LOADING=EAGER, if device memory may run out later.
 *  - Synchronises `stream` and returns FQ_EBOUND if the device check fired.
 *  - Every call shares the array and overwrites what the previous call left there; calls
 *    that overlap on the GPU (other streams, other host threads) race and must not be made. */
fq_status floquet_build_UT_static(const fq_problem* problem, void* d_U, void* stream);

/* Batched scan (many independent problems, one launch; the paper's method applied to a scan of
 * drive parameters).  Plan i writes d_U[i] (its N_i x N_i complex128 U_T, as floquet_build_UT)
 * and floquet_batch_launch replays the whole scan as one graph launch on `stream`.
 *  - lanes = 0: when every plan is a split-precision dense plan (FQ_BF16X3 or FQ_BF16X6, Magnus
 *    order 4, L <= 32) of one precision and one step count M, the graph holds ONE persistent
 *    tensor-core kernel (one CTA per SM) whose CTAs take work units from a device counter: per
 *    instance the blocks of Omega~_m's slices (Eqs. 11 and 14), and per step, term and output
 *    tile the Chebyshev term of Eq. 10 (state blocks of 128 columns advance independently, each
 *    unit waiting, with a bounded spin, only for the units it reads).  The tile width is the one
 *    the plans' own widths favour (tile_n or floquet_autotune), weighted by N^3 M L, with the
 *    width's default K stage; each U_T then equals the plan's own floquet_build_UT bit for bit
 *    when the tile shapes agree.  Other plans fall back to 8 lanes.
 *  - lanes = 1..32: floquet_build_UT of every plan captured on `lanes` concurrent graph
 *    branches, assigned longest-first by their cost N^3 M L.
 *  - A wait that gives up marks every plan's status word FQ_BIT_TIMEOUT (floquet_check_status
 *    reports FQ_ETIMEOUT); the device check marks the plan it fired for.
 * The plans, outputs and workspace must outlive the batch; the graph is bound to those pointers,
 * and the batch's launches must not overlap one another on the GPU (they share the workspace).
 * Creating the batch enqueues nothing (lanes = 0 writes its unit tables into d_ws with a
 * synchronous copy).
 * d_ws: floquet_batch_workspace_size(plans, count) bytes, 256-byte aligned (it includes the
 * persistent scan's tables, counters and second Omega~ buffers when the plans qualify). */
typedef struct fq_batch fq_batch;
size_t floquet_batch_workspace_size(fq_plan* const* plans, int32_t count);
fq_status floquet_batch_create(fq_batch** batch, fq_plan* const* plans, int32_t count, void* const* d_U,
                               void* d_ws, size_t ws_bytes, int32_t lanes);
fq_status floquet_batch_launch(fq_batch* batch, void* stream);
void floquet_batch_destroy(fq_batch* batch);

/* Autotuner for the split-precision dense path: times each tile shape of the tensor-core term
 * kernel on two steps of this plan (states: the identity block) and keeps the fastest for the
 * plan's later calls.  Shapes: output widths 64 and 128 (K stages of 32 elements, 64 for 64-wide
 * BF16X3 tiles), and for BF16X3 also 64-wide tiles with 32-element K stages; each runs as many
 * stages as fit in shared memory.  d_ws as for floquet_build_UT.  Synchronises `stream`; no-op
 * (FQ_OK) for other paths.  *tile_n receives the chosen width (NULL allowed); on an error the plan
 * keeps the shape it had. */
fq_status floquet_autotune(fq_plan* plan, void* d_ws, size_t ws_bytes, void* stream, int32_t* tile_n);

/* Synchronises `stream`; returns FQ_ETIMEOUT if a bounded device wait of this plan's kernels
 * gave up, else FQ_EBOUND if a numerical device check fired, since the last call (and clears
 * the word); FQ_OK otherwise. */
fq_status floquet_check_status(fq_plan* plan, void* stream);

/* Diagnostic of the timeout path: one thread waits, bounded by `cycles` SM clock cycles (at most
 * 2^31), on a shared-memory mbarrier that nothing arrives on, exactly as the tensor-core
 * kernels wait on their pipeline barriers, then records the timeout in the plan's status word
 * and returns.  The next floquet_check_status reports FQ_ETIMEOUT; the context stays usable. */
fq_status floquet_selftest_wait(fq_plan* plan, int64_t cycles, void* stream);

/* FP32 rate probe, a measurement aid (the paper has no counterpart): one launch of min(4 x SMs,
 * out_len / 256) CTAs of 256 threads, each thread running independent chains of `iters` fused
 * multiply-adds, packed over lane pairs (FFMA2, packed != 0) or scalar, enqueued on `stream`.
 * d_out: caller-owned device buffer of out_len floats (one sum per thread is written).  *flops
 * receives the launch's flop count (2 per multiply-add), so a caller timing the launch with CUDA
 * events gets the GPU's sustained FP32 rate.  FQ_EINVAL for iters < 1, NULL pointers or
 * out_len < 256. */
fq_status floquet_probe_fp32(int32_t packed, int32_t iters, float* d_out, int64_t out_len, void* stream,
                             double* flops);

/* Quasienergies (Eq. 5) and Floquet states of U_T on the host, outside the timed propagation:
 * U = N x N complex128 host array, row-major, U[i][j] = <i|U_T|j> (as floquet_build_UT writes it).
 * eps_out: N doubles, eps_mu = theta_mu / T with theta_mu = -arg(lambda_mu) folded into
 * [-pi, pi), ascending.  states_out (NULL: not computed): N x N complex128, row mu = the unit
 * Floquet state of eps_out[mu].  Complex Schur form by Householder reduction and shifted QR
 * (no LAPACK linked; O(N^3) on up to 16 host threads: about 3.5 s at N = 1000 for eps alone,
 * 4.7 s with the states, on 8 cores); U_T is normal, so the Schur vectors are its eigenvectors.
 * Safe to call from several host threads at once.  FQ_EINVAL on bad
 * arguments or if the iteration does not converge.  Needs no device; every array is the caller's. */
fq_status floquet_quasienergies(const void* U, int32_t n, double period, double* eps_out, void* states_out);

/* Message of the last failing call on this thread ("" if none). */
const char* floquet_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FLOQUET_H */
