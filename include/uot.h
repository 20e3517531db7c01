/*
 * uot.h -- C ABI of libuot: entropic unbalanced optimal transport with
 * rho*KL marginal penalties on one GB300 (sm_103a), solved by log-domain
 * Sinkhorn and by translation-invariant Sinkhorn (H-Sinkhorn, also G-Sinkhorn
 * and Anderson extrapolation), and, for 1-D problems at eps = 0, by
 * Frank-Wolfe on the translation-invariant functional (uot_fw1d_batched).
 *
 * Method: Sejourne, Vialard, Peyre, "Faster Unbalanced Optimal Transport:
 * Translation invariant Sinkhorn and 1-D Frank-Wolfe" (AISTATS 2022).
 *
 *   primal  UOT(a,b) = min_{pi>=0} <pi,C> + eps KL(pi|a(x)b)
 *                      + rho1 KL(pi 1|a) + rho2 KL(pi^T 1|b)      Sec. 1, Eq. (eq-primal-uot-kl)
 *   dual    F_eps(f,g) = <a, rho1(1-e^{-f/rho1})> + <b, rho2(1-e^{-g/rho2})>
 *                      - eps <a(x)b, e^{(f(+)g-C)/eps} - 1>       Sec. 1, Eq. (eq-dual-uot-kl)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - f, x, a, rho1 and index i (N of them) form one side; g, y, b, rho2 and
 *    index j (M of them) the other.  C is N x M.
 *  - All data pointers are DEVICE pointers on the current CUDA device and are
 *    owned by the caller: inputs, outputs and the workspace.  The library
 *    allocates no device memory.
 *  - Float data is FP32, row-major and contiguous: x is N x dim, y is M x dim,
 *    C is N x M.  Weights may contain zeros (those points drop out of every
 *    sum) but no negative, NaN or infinite entries, and each side needs at
 *    least one positive weight; such data errors are detected on the device
 *    and reported as UOT_ERR_NONFINITE.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it.  uot_sinkhorn and uot_ti_sinkhorn synchronise the stream
 *    at every residual check (they decide on the host when to stop) and on
 *    return; the other calls are asynchronous.
 *  - `ws` is a device workspace of at least uot_workspace_size() bytes,
 *    256-byte aligned.  Calls sharing a workspace must not overlap in time.
 *  - Argument errors are detected on the host before anything is enqueued;
 *    the call then returns UOT_ERR_INVALID_ARG / UOT_ERR_WORKSPACE /
 *    UOT_ERR_UNSUPPORTED and uot_last_error() describes the problem.
 *  - No exception, abort or device trap crosses this interface.
 */
#ifndef UOT_H
#define UOT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define UOT_API __attribute__((visibility("default")))
#else
#define UOT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  UOT_OK = 0,
  UOT_ERR_INVALID_ARG = 1,  /* bad size, parameter or pointer                   */
  UOT_ERR_WORKSPACE = 2,    /* workspace missing, too small or misaligned       */
  UOT_ERR_CUDA = 3,         /* a CUDA runtime call failed (see uot_last_error)  */
  UOT_ERR_NONFINITE = 4,    /* NaN/Inf met on the device, or invalid weights    */
  UOT_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up               */
  UOT_NOT_CONVERGED = 6,    /* max_iter reached above tol; outputs are valid    */
  UOT_ERR_UNSUPPORTED = 7   /* valid request this build does not implement      */
} uot_status;

typedef enum { UOT_COST_POINTS = 0, UOT_COST_DENSE = 1 } uot_cost_kind;

/* One problem.  Cost C_ij = |x_i - y_j|_2^p (points, computed on the fly and
 * never stored; Sec. 1 and the 1-D experiments of Sec. 4) or a stored matrix
 * (dense).  eps, rho1, rho2 > 0 and finite (Sec. 1). */
typedef struct {
  int32_t n, m;        /* N >= 1 rows (x, a, f), M >= 1 columns (y, b, g)           */
  int32_t dim;         /* point dimension, 1..64 (points); ignored for dense          */
  int32_t cost_kind;   /* uot_cost_kind                                               */
  float p;             /* exponent p >= 1 of the points cost; p == 2 is the fast path */
  int32_t ordering;    /* points cost with dim <= 3 and p == 2 only: 0 = automatic, 1 = always put  */
                       /* both clouds in Morton order and use the tiled sweeps, 2 = never.          */
                       /* Results agree within rounding; ordering costs a few hundred us per call   */
                       /* and pays off from about 1.5e9 cost entries per call, the automatic        */
                       /* threshold.  With 0, a solve of a problem with N M <= 2^20 whose clouds    */
                       /* fit one SM's shared memory (16 N + 20 M + 12 max(N, M) bytes plus 8 (1-D) */
                       /* or 16 bytes per point, <= 200 KB) runs the whole loop in one launch of a  */
                       /* thread-block cluster instead (no ordering).                               */
  double eps, rho1, rho2;
  const float* x;      /* device, N x dim (points)        */
  const float* y;      /* device, M x dim (points)        */
  const float* C;      /* device, N x M (dense)           */
  const float* a;      /* device, N weights, a_i >= 0      */
  const float* b;      /* device, M weights, b_j >= 0      */
} uot_problem;

/* Divergence of a marginal penalty for uot_sinkhorn_phi (Sec. 3): the convex
 * conjugate phi^* of the penalty, with parameter rho (rho1 for a, rho2 for b). */
typedef enum {
  UOT_PHI_KL = 0,   /* rho KL:        phi^*(q) = rho (e^{q/rho} - 1)          */
  UOT_PHI_BERG = 1  /* Berg entropy:  phi^*(q) = -rho log(1 - q/rho), q < rho */
} uot_phi;

/* Iteration control for uot_sinkhorn / uot_ti_sinkhorn / uot_g_sinkhorn. */
typedef struct {
  int32_t max_iter;          /* >= 1 full iterations (g half-step, then f half-step)          */
  int32_t check_every;       /* >= 1: residual tested against tol every check_every iterations */
  double tol;                /* >= 0 fixed-point residual tolerance in cost units; 0 = run     */
                             /* exactly max_iter iterations                                      */
  int32_t warm_start;        /* nonzero: f holds the initial potential on entry                 */
  int32_t lse_reference;     /* tiled sweeps of uot_sinkhorn / uot_ti_sinkhorn (Morton-ordered   */
                             /* clouds): each row's log-sum-exp of the previous iteration may    */
                             /* serve as the fixed exponent reference of the next one, which     */
                             /* removes the running max from the inner loop.  0 = automatic     */
                             /* (once the largest change between two iterations is below 24     */
                             /* in log2 units), 1 = never, 2 = from the second iteration on.    */
                             /* Rows that land outside a +-60 window around their reference are */
                             /* recomputed exactly, so every setting gives the same result       */
                             /* within rounding; only the time differs.  Other paths ignore it. */
  float* residual_history;   /* device, nullable, >= max_iter+1 floats: entry t is the residual */
                             /* of iterate t (t = 1..iters); entry 0 is unused                   */
  /* Anderson extrapolation (appendix, "Combining Sinkhorn with Anderson acceleration"),     */
  /* uot_sinkhorn / uot_ti_sinkhorn / uot_g_sinkhorn.  The iterate x is f, fb or fb (with      */
  /* lambda carried alongside) respectively; after every anderson_k-th iteration t, unless t   */
  /* is the last one or a residual check, the last anderson_k + 1 iterates x_{t-K}..x_t are     */
  /* replaced by sum_{k<K} c_k x_{t-K+k}, c = (G + r I)^{-1} 1 / 1^T (G + r I)^{-1} 1, with      */
  /* G = U^T U / trace(U^T U) for the residuals u_k = x_{t-K+k+1} - x_{t-K+k} (FP64, on the    */
  /* device), which starts the next block.  The returned pair is always a plain iterate's.   */
  int32_t anderson_k;        /* 0 = off, else K in 2..6                                        */
  double anderson_reg;       /* r >= 0 (the paper's experiment: 1e-7)                          */
  void* anderson_buf;        /* device, >= uot_anderson_workspace(n, anderson_k) bytes, 16-byte */
                             /* aligned, when anderson_k > 0; caller-owned scratch              */
} uot_options;

/* Bytes of the scratch uot_options.anderson_buf needs for N = n and K = k. */
UOT_API size_t uot_anderson_workspace(int32_t n, int32_t k);

/* Outcome of a solve, written to host memory before the call returns. */
typedef struct {
  int32_t iters;       /* index T of the returned iterate                                   */
  int32_t converged;   /* 1 if residual <= tol                                              */
  int32_t status;      /* uot_status of the solve                                           */
  int32_t lse_misses;  /* rows recomputed after their fixed reference missed (lse_reference) */
  double residual;     /* fixed-point residual of the returned (f, g), see below            */
  double lambda;       /* TI: lambda*(fb_T, gb_T) of Prop. 2; plain: 0                      */
} uot_result;

/* Bytes of device workspace needed by any entry point on `prob` (0 on an
 * invalid problem; uot_last_error() then says why).  Depends on the problem's
 * sizes, dim, cost kind and on the current device's SM count. */
UOT_API size_t uot_workspace_size(const uot_problem* prob);

/* Row or column softmin sweep, the O(NM) primitive of every Sinkhorn variant
 * (Sec. 3, definition of Smin):
 *   axis 0: out_i = Smin_b^eps(C(x_i,.) - pot) = -eps log sum_j b_j exp((pot_j - C_ij)/eps),
 *           pot and out are M- and N-vectors;
 *   axis 1: out_j = Smin_a^eps(C(.,y_j) - pot) = -eps log sum_i a_i exp((pot_i - C_ij)/eps),
 *           pot and out are N- and M-vectors.
 * Asynchronous. */
UOT_API uot_status uot_softmin(const uot_problem* prob, int32_t axis, const float* pot, float* out,
                       void* ws, size_t ws_bytes, void* stream);

/* The same sweep as uot_softmin for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a deployment variant.
 *
 * Some callers have no device allocator at hand (a plain C host program
 * without a memory pool, a plug-in whose host framework forbids allocation
 * after start-up, a real-time loop that must not call cudaMalloc).  This entry
 * point takes no workspace: its scratch is a 32 MiB array compiled into the
 * library, reserved on every GPU that loads the library's device code and held
 * until the process exits.  The call itself performs no cudaMalloc, cudaFree
 * or other allocation.
 *  - Limit: problems whose uot_workspace_size() exceeds 32 MiB are rejected
 *    with UOT_ERR_UNSUPPORTED and a message; use uot_softmin for those.  With
 *    N = M and 3-D points on a 152-SM GB300, 70000 points per side fit and
 *    80000 do not (the partial buffers follow the launch shapes, so the size
 *    does not grow smoothly with N).
 *  - The first call on each device looks up the scratch's device address with
 *    that device current; make that first call before any stream capture.
 *    Under lazy module loading (CUDA_MODULE_LOADING=LAZY, CUDA's default) that
 *    first call is also where the driver loads this library's device code and
 *    reserves the 32 MiB, so it is the one call that can fail with
 *    UOT_ERR_CUDA for lack of device memory: callers that must not fail later
 *    (real-time loops) should make one warm-up call during start-up.  After
 *    cudaDeviceReset the look-up is redone on the next call (the address is
 *    cached per device and per CUDA context).
 *  - All calls share the one scratch array, which keeps the last call's
 *    contents (every call resets the parts it reads before reading them).
 *    Calls whose GPU work overlaps in time (two host threads, or two streams
 *    on the same device) race on the scratch and give wrong results: serialise
 *    them.
 * Arguments and results as for uot_softmin.  Asynchronous. */
UOT_API uot_status uot_softmin_noalloc(const uot_problem* prob, int32_t axis, const float* pot, float* out,
                                       void* stream);

/* Plain (F-)Sinkhorn, Sec. 3:
 *   g_{t+1} = rho2/(rho2+eps) Smin_a^eps(C - f_t),  f_{t+1} = rho1/(rho1+eps) Smin_b^eps(C - g_{t+1}),
 * from f_0 = 0 (or f on entry when warm_start).  On return f, g hold (f_T, g_T).
 * The residual is the sup-norm violation of the F-Sinkhorn fixed-point
 * equations by the returned pair (cost units):
 *   r = max(|f - rho1/(rho1+eps) Smin_b^eps(C - g)|_inf, |g - rho2/(rho2+eps) Smin_a^eps(C - f)|_inf);
 * the first term is zero up to rounding because f is computed from g, so the
 * library evaluates the second, which costs one more column sweep at exit.
 * Returns UOT_OK, UOT_NOT_CONVERGED (outputs valid) or an error. */
UOT_API uot_status uot_sinkhorn(const uot_problem* prob, const uot_options* opt, float* f, float* g,
                        uot_result* result, void* ws, size_t ws_bytes, void* stream);

/* Translation-invariant Sinkhorn = H-Sinkhorn (Sec. 3, Prop. 4; general
 * rho1 != rho2 from the proof of Prop. 4 in App. B):
 *   g_hat = rho2/(rho2+eps) Smin_a^eps(C - fb) - eps/(eps+rho2) rho2/(rho1+rho2) Smin_a^rho1(fb)
 *   gb    = g_hat + k_g/(1-k_g) Smin_b^rho2(g_hat),   k_g = eps/(eps+rho2) rho1/(rho1+rho2)
 * and symmetrically for fb, from fb_0 = 0 (or f on entry).
 * Precision: the softmin sweeps are FP32.  The two mass reductions Smin^rho,
 * their logs, the closed-form translation and lambda* (Prop. 2) run in
 * float-pair arithmetic (two floats, ~2^-44 relative per operation; FP64 is
 * ~64x slower than FP32 on this GPU and these scalars sit on every half-step's
 * critical path); a reduction of 262144 terms agrees with a long-double sum of
 * the same terms to better than 1e-10 relative, far below the FP32 rounding of
 * the potentials that enter it.  FP64 copies of the scalars are kept for the
 * host (result->lambda) and for the O(N + M) kernels.
 * On return f, g hold (f, g) = Phi(fb_T, gb_T) = (fb_T + lambda*, gb_T - lambda*).
 * Residual as for uot_sinkhorn, on the translated pair. */
UOT_API uot_status uot_ti_sinkhorn(const uot_problem* prob, const uot_options* opt, float* f, float* g,
                           uot_result* result, void* ws, size_t ws_bytes, void* stream);

/* G-Sinkhorn (Sec. 3): alternate maximisation of G(fb, gb, lambda), with the
 * translation lambda* of Prop. 2 refreshed after every full iteration:
 *   gb_{t+1} = rho2/(rho2+eps) Smin_a^eps(C - fb_t - lambda_t) + lambda_t
 *   fb_{t+1} = rho1/(rho1+eps) Smin_b^eps(C - gb_{t+1} + lambda_t) - lambda_t
 *   lambda_{t+1} = lambda*(fb_{t+1}, gb_{t+1})
 * from fb_0 = 0 (or f on entry), lambda_0 = 0.  The mass reductions behind
 * lambda* are float-pair sums (~1e-11 relative).  On return f, g hold
 * (fb_T + lambda_T, gb_T - lambda_T) and result->lambda = lambda_T.  The
 * residual is that of uot_sinkhorn on the returned pair, which equals
 * |gb_{T+1} - gb_T|_inf.  Arguments, results and errors as for
 * uot_ti_sinkhorn. */
UOT_API uot_status uot_g_sinkhorn(const uot_problem* prob, const uot_options* opt, float* f, float* g,
                          uot_result* result, void* ws, size_t ws_bytes, void* stream);

/* Plans: a solve with no host synchronisation, capturable in a CUDA graph.
 *
 * uot_plan_create fixes a problem (its sizes, parameters and device pointers),
 * its options and the variant (0: plain F-Sinkhorn as uot_sinkhorn, 1:
 * H-Sinkhorn as uot_ti_sinkhorn, 2: G-Sinkhorn as uot_g_sinkhorn; Sec. 3).
 * uot_plan_solve then enqueues the whole solve on `stream` and returns at
 * once: the iterations run as a CUDA graph whose loop is a conditional while
 * node, the stopping rule of uot_sinkhorn (residual tested every check_every
 * iterations and at max_iter) evaluated on the device after each g half-step,
 * so the host never waits.  The same iterates, residual and result as the
 * host-driven entry points (equal within rounding of the same kernels).
 *  - res_dev: DEVICE memory for one uot_result, written at the end of the
 *    solve (read it after synchronising the stream); its status field holds
 *    the solve's uot_status (UOT_OK, UOT_NOT_CONVERGED, UOT_ERR_NONFINITE,
 *    UOT_ERR_TIMEOUT).  The call's own return value reports argument and CUDA
 *    errors only.
 *  - If `stream` is being captured (cudaStreamBeginCapture), the solve is
 *    added to the caller's graph (with its conditional nodes) and replays with
 *    it.  Otherwise the library captures the solve once per set of (f, g,
 *    res_dev, ws) pointers into an executable graph kept in the plan (the last
 *    four) and launches it.  Buffers are read when the solve runs, so their
 *    contents may change between solves; the problem's device pointers must
 *    stay valid while the plan is used.
 *  - Workspace: uot_plan_workspace_size(plan) bytes, as for uot_workspace_size.
 *  - Anderson extrapolation (options.anderson_k) is host-driven and rejected
 *    here with UOT_ERR_UNSUPPORTED; options.residual_history works (entry t is
 *    written by the solve on the device).
 *  - A plan belongs to the device that was current at creation; calls on one
 *    plan are serialised (a mutex) and solves sharing a workspace must not
 *    overlap on the GPU.  uot_plan_create allocates host memory and three CUDA
 *    streams, no device memory; uot_plan_destroy releases them. */
typedef struct uot_plan uot_plan;
UOT_API uot_status uot_plan_create(const uot_problem* prob, const uot_options* opt, int32_t variant,
                                   uot_plan** out);
UOT_API void uot_plan_destroy(uot_plan* plan);
UOT_API size_t uot_plan_workspace_size(const uot_plan* plan);
UOT_API uot_status uot_plan_solve(uot_plan* plan, float* f, float* g, uot_result* res_dev, void* ws,
                                  size_t ws_bytes, void* stream);

/* Dual objective F_eps(f, g) (Sec. 1, Eq. eq-dual-uot-kl), FP64, written to
 * out[0] (device).  If out has room for 3 doubles (want_primal != 0) it also
 * writes out[1] = primal objective (Eq. eq-primal-uot-kl) of the plan
 * pi_ij = a_i b_j e^{(f_i+g_j-C_ij)/eps} and out[2] = m(pi); at the optimum
 * out[0] == out[1] (zero duality gap).  One row sweep (two with the primal)
 * plus O(N+M) FP64 reductions.  Asynchronous. */
UOT_API uot_status uot_dual_value(const uot_problem* prob, const float* f, const float* g, double* out,
                          int32_t want_primal, void* ws, size_t ws_bytes, void* stream);

/* Gradient of UOT = F_eps(f*, g*) with respect to a, b, x, y by the envelope
 * theorem (used by the paper in the proof of Prop. 1): the partial
 * derivatives of F_eps at the given (f, g), which should be the optimal pair:
 *   grad_a_i = rho1 (1 - e^{-f_i/rho1}) - eps (e^{(f_i - S_i)/eps} - m(b)),  S = Smin_b^eps(C - g)
 *   grad_b_j = rho2 (1 - e^{-g_j/rho2}) - eps (e^{(g_j - S'_j)/eps} - m(a)), S' = Smin_a^eps(C - f)
 *   grad_x_i = sum_j pi_ij dC_ij/dx_i,   grad_y_j = sum_i pi_ij dC_ij/dy_j,
 * with pi formed on the fly and never stored.  Each output pointer may be NULL
 * (not computed); grad_x / grad_y need the points cost.  Asynchronous (nothing is read back: for dim >=
 * 32 a bounded tensor-core wait that gives up leaves NaN in the gradients). */
UOT_API uot_status uot_grad(const uot_problem* prob, const float* f, const float* g, float* grad_a,
                    float* grad_b, float* grad_x, float* grad_y, void* ws, size_t ws_bytes,
                    void* stream);

/* Measurement hooks (no counterpart in the paper).
 * uot_kernel_launches: number of CUDA kernels this library has launched in the
 * process so far (all threads).
 * uot_profile_begin / uot_profile_end: while a profile is open on the calling
 * thread, every softmin sweep kernel launched by that thread is bracketed by a
 * pair of CUDA events recorded on its launch stream (at most 65536 launches are
 * bracketed; later ones are counted but not timed).  uot_profile_end
 * synchronises those events and returns the summed device time of the timed
 * sweep launches in *sweep_ms, their number in *timed_launches and the number of
 * sweep launches seen in *launches.  Events are created at begin and destroyed
 * at end.  Returns UOT_ERR_INVALID_ARG when no profile is open. */
UOT_API uint64_t uot_kernel_launches(void);
/* Test hook (no counterpart in the paper): caps the number of polls of the
 * main-loop mbarrier waits of the tensor-core sweeps (dim <= 3 tiled solver
 * half-steps, dim >= 32 sweeps) at `polls` (0 restores the default, about
 * 1.7e7; a negative value allows no poll at all), process-wide, for launches
 * made afterwards.  With no poll allowed every such wait gives up at once
 * (with one poll, only those whose condition is not met within the first
 * poll's wait window): the sweep then stops its roles, lets every
 * copy and MMA in flight land (those waits keep the default limit), frees its
 * tensor memory and reports a timeout, so that the solver returns
 * UOT_ERR_TIMEOUT and the CUDA context stays usable.  This is how the timeout
 * path is tested without faulting or hanging a GPU. */
UOT_API void uot_test_set_wait_limit(int64_t polls);
UOT_API uot_status uot_profile_begin(void);
UOT_API uot_status uot_profile_end(double* sweep_ms, int64_t* timed_launches, int64_t* launches);

/* Unrolled gradient of the truncated solve: with (f_T, g_T) = Phi(fb_T, gb_T)
 * after T H-Sinkhorn iterations from fb_0 = 0 (as uot_ti_sinkhorn with
 * max_iter = T, tol = 0), writes value[0] = F_eps(f_T, g_T) (device double) and
 * the exact derivatives of that value with respect to a, b, x, y (outputs
 * nullable), obtained by reverse mode through all T iterations: each half-step
 * (softmin sweep, aprox, FP64 mass reduction and translation of the proof of
 * Prop. 4, App. B) is differentiated, the softmins by one adjoint sweep each.
 * Iterates are checkpointed every ckpt_every iterations and each segment is
 * recomputed once during the reverse pass (memory O((N + M) (T/ckpt_every +
 * ckpt_every (dim + 3)))).  Points cost with p = 2 only.  Workspace:
 * uot_unrolled_workspace_size.  Synchronises the stream on return. */
UOT_API size_t uot_unrolled_workspace_size(const uot_problem* prob, int32_t T, int32_t ckpt_every);
UOT_API uot_status uot_grad_unrolled(const uot_problem* prob, int32_t T, int32_t ckpt_every, double* value,
                                     float* grad_a, float* grad_b, float* grad_x, float* grad_y, void* ws,
                                     size_t ws_bytes, void* stream);

/* A batch of independent problems with the points cost |x - y|^2 (p = 2) and
 * dim <= 3, each with its own sizes, dimension and parameters.  Data of all
 * problems is packed in shared device arrays; offsets are element offsets into
 * those arrays.  f and g outputs use the offsets of a and b. */
typedef struct {
  int32_t count;          /* number of problems >= 1                                      */
  int32_t reserved;
  const int32_t* n;       /* host [count]: N_k >= 1                                        */
  const int32_t* m;       /* host [count]: M_k >= 1                                        */
  const int32_t* dim;     /* host [count]: 1..3                                            */
  const double* eps;      /* host [count]                                                  */
  const double* rho1;     /* host [count]                                                  */
  const double* rho2;     /* host [count]                                                  */
  const int64_t* x_off;   /* host [count]: first coordinate of problem k in x (N_k x dim_k) */
  const int64_t* y_off;   /* host [count]: first coordinate of problem k in y              */
  const int64_t* a_off;   /* host [count]: first weight of problem k in a (and f)          */
  const int64_t* b_off;   /* host [count]: first weight of problem k in b (and g)          */
  const float* x;         /* device, packed coordinates                                    */
  const float* y;
  const float* a;         /* device, packed weights                                        */
  const float* b;
} uot_batch;

/* Workspace bytes for uot_sinkhorn_batched on `batch` (0 if invalid). */
UOT_API size_t uot_batch_workspace_size(const uot_batch* batch);

/* Plain (ti = 0) or translation-invariant (ti = 1) Sinkhorn on every problem of
 * the batch at once (same updates, residual and stopping rule per problem as
 * uot_sinkhorn / uot_ti_sinkhorn; opt->warm_start and residual_history are not
 * supported and must be 0 / NULL).  Each half-step is one launch over all
 * problems still running; problems stop individually when their residual is
 * <= tol at a check, or at max_iter.  With a non-NULL stream, chunks of
 * check_every iterations are captured once as a CUDA graph and replayed.
 * results: host [count], filled before return.  Returns UOT_OK when every
 * problem converged, UOT_NOT_CONVERGED when some stopped at max_iter, an
 * error otherwise. */
UOT_API uot_status uot_sinkhorn_batched(const uot_batch* batch, const uot_options* opt, int32_t ti, float* f,
                                        float* g, uot_result* results, void* ws, size_t ws_bytes, void* stream);

/* 1-D unregularised UOT (eps = 0, rho_i KL penalties) by Frank-Wolfe on the
 * translation-invariant functional H_0 (Sec. 4, Alg. 2) for a batch of
 * independent problems.  Each step computes lambda*(fb, gb) (Prop. 2), the
 * re-weighted histograms a~ = a e^{-(fb + lambda*)/rho1},
 * b~ = b e^{-(gb - lambda*)/rho2} (Eq. fw-updated-histo, equal masses by
 * Prop. 1), the exact balanced 1-D OT duals (r, s) between them by one walk
 * over the sorted points (SolveOT1D, Alg. 1, read as the north-west corner
 * rule: the point whose remaining mass is smaller is exhausted first), and
 * (fb, gb) <- (1 - gamma_t)(fb, gb) + gamma_t (r, s) with gamma_t = 2/(2 + t),
 * from (fb, gb) = 0.  Outputs the translated pair (fb + lambda*, gb - lambda*).
 * Cost |x_i - y_j|^p.  lambda*, the histograms, the walk's mass bookkeeping
 * (hence its branches) and the step are FP64 on the device; the walk's
 * potentials are float pairs (about 2^-44 relative per operation).  One warp
 * runs one problem. */
typedef struct {
  int32_t count;          /* number of problems >= 1                                      */
  int32_t n_iter;         /* Frank-Wolfe steps >= 1                                       */
  double p;               /* cost exponent, finite and >= 1, shared by the batch          */
  const int32_t* n;       /* host [count]: N_k >= 1                                        */
  const int32_t* m;       /* host [count]: M_k >= 1                                        */
  const int64_t* x_off;   /* host [count]: first point of problem k in x, a and f (>= 0)   */
  const int64_t* y_off;   /* host [count]: first point of problem k in y, b and g (>= 0)   */
  const double* rho1;     /* host [count]: finite, > 0                                     */
  const double* rho2;     /* host [count]: finite, > 0                                     */
  const float* x;         /* device, packed; ascending within each problem                */
  const float* a;         /* device, packed weights >= 0, positive total per problem      */
  const float* y;
  const float* b;
} uot_fw1d_batch;

/* Workspace bytes for uot_fw1d_batched on `batch` (0 if the batch is invalid;
 * uot_last_error() says why). */
UOT_API size_t uot_fw1d_workspace_size(const uot_fw1d_batch* batch);

/* Runs batch->n_iter Frank-Wolfe steps on every problem.  f, g: device FP64
 * outputs indexed like a and b (problems must not overlap there).  status:
 * optional host [count], per problem UOT_OK, UOT_ERR_INVALID_ARG (points not
 * ascending or not finite) or UOT_ERR_NONFINITE (a weight negative or not
 * finite, or a side's total mass zero); such a problem's outputs are NaN.
 * Host-side checks (sizes, parameters, pointers, workspace: 256-byte aligned,
 * at least uot_fw1d_workspace_size bytes) fail before any device work.
 * Synchronises the stream; returns UOT_OK when every problem is valid, else
 * the first failing problem's status. */
UOT_API uot_status uot_fw1d_batched(const uot_fw1d_batch* batch, double* f, double* g, int32_t* status,
                                    void* ws, size_t ws_bytes, void* stream);

/* 1-D unbalanced multi-marginal OT and barycenters (Sec. 5): K measures
 * (x_k, alpha_k) on the line per problem, barycentric weights omega_k > 0
 * summing to one, rho KL penalties (rho_k = omega_k rho in the dual) and the
 * squared-distance cost, whose multi-marginal form is
 *   C(z_1..z_K) = sum_k omega_k (z_k - B(z))^2,  B(z) = sum_k omega_k z_k.
 * Frank-Wolfe on the translation-invariant functional H: each step computes
 * the optimal translation lambda (Sec. 5, rho KL setting:
 * lambda_k = omega_k rho q_k - omega_k sum_l omega_l rho q_l / sum_l omega_l,
 * q_k = log <alpha_k, e^{-fb_k/(omega_k rho)}>), the re-weighted measures
 * alpha~_k = alpha_k e^{-(fb_k + lambda_k)/(omega_k rho)}, the balanced
 * multi-marginal duals r between them by one pass over the sorted points
 * (SolveMOT, Alg. 3: the measure with the least remaining mass among those
 * not at their last point moves, lowest index on ties; the last index tuple
 * takes the mass left), and fb <- (1 - tau_t) fb + tau_t r, tau_t = 2/(2+t),
 * from fb = 0.  Outputs the translated potentials f_k = fb_k + lambda_k and the
 * barycenter of Prop. prop:barycentermulti: the points B(tuple) of the plan
 * SolveMOT returns at the final iterate (tuples of positive mass, in plan
 * order) with those masses as weights.  FP64 throughout; one warp runs one
 * problem. */
typedef struct {
  int32_t count;          /* number of problems >= 1                                           */
  int32_t n_iter;         /* Frank-Wolfe steps >= 1                                            */
  int32_t K;              /* measures per problem, 2..8, shared by the batch                    */
  int32_t reserved;
  const int32_t* n;       /* host [count * K]: points of measure k of problem p at [p * K + k]  */
  const int64_t* off;     /* host [count * K]: first point of that measure in x, alpha and f    */
  const double* rho;      /* host [count]: finite, > 0                                         */
  const double* omega;    /* host [count * K]: barycentric weights > 0, summing to one          */
  const float* x;         /* device, packed points, ascending within each measure             */
  const float* alpha;     /* device, packed weights >= 0, positive total per measure          */
} uot_mmot1d_batch;

/* Workspace bytes of uot_mmot1d_batched (0 if the batch is invalid), and the
 * length of the barycenter output arrays: the sum over problems of their
 * points, problem p's barycenter starting after those of problems 0..p-1. */
UOT_API size_t uot_mmot1d_workspace_size(const uot_mmot1d_batch* batch);
UOT_API size_t uot_mmot1d_barycenter_size(const uot_mmot1d_batch* batch);

/* Runs batch->n_iter Frank-Wolfe steps on every problem.  f: device FP64,
 * indexed like x.  bary_x, bary_w: device FP64 of uot_mmot1d_barycenter_size
 * entries; bary_len: optional host [count], the number of barycenter points of
 * each problem.  status: optional host [count], per problem UOT_OK,
 * UOT_ERR_INVALID_ARG (points not ascending or not finite) or
 * UOT_ERR_NONFINITE (a weight negative or not finite, or a measure of zero
 * mass).  Synchronises the stream; returns UOT_OK when every problem is valid,
 * else the first failing problem's status. */
UOT_API uot_status uot_mmot1d_batched(const uot_mmot1d_batch* batch, double* f, double* bary_x, double* bary_w,
                                      int32_t* bary_len, int32_t* status, void* ws, size_t ws_bytes, void* stream);

/* F- and G-Sinkhorn for a general smooth phi^* (Sec. 3), phi1 for the
 * penalty on a, phi2 for the one on b (uot_phi).  With
 * aprox_{phi^*}(x) = argmin_y eps e^{(x - y)/eps} + phi^*(y), one iteration is
 *   variant 0 (F):  g <- -aprox_2(-Smin_a(C - f)),            f <- -aprox_1(-Smin_b(C - g));
 *   variant 2 (G):  gb <- -aprox_2(-Smin_a(C - fb - lambda)) + lambda,
 *                   fb <- -aprox_1(-Smin_b(C - gb + lambda)) - lambda,  lambda <- lambda*(fb, gb),
 * lambda* = argmax_l <a, -phi_1^*(-fb - l)> + <b, -phi_2^*(-gb + l)> (Prop. 1),
 * from f_0 = 0 (or f on entry with warm_start; G starts from fb_0 = f, lambda_0 = 0).
 * The softmins run on the sweeps of uot_softmin (FP32, the 1e-4 eps bound);
 * the prox maps and lambda* in FP64 (Berg: aprox(x) = rho - eps omega(L),
 * omega the Wright omega function, L = log(rho/eps) + (rho - x)/eps; lambda* by
 * Newton steps kept inside a bracket of the root).  Returns f (= fb + lambda for G)
 * and g (= gb - lambda), result->lambda = lambda (0 for F), result->residual =
 * max_j |g_t - g_{t-1}| of the last iteration (gb for G), tested every
 * check_every iterations against opt->tol.  Options anderson_k and
 * residual_history are not used; lse_reference has no effect.  Workspace:
 * uot_sinkhorn_phi_workspace_size(prob) bytes, 256-byte aligned.  Errors as for
 * uot_sinkhorn, plus UOT_ERR_INVALID_ARG for another variant or divergence.
 * With phi1 = phi2 = UOT_PHI_KL, variant 0 gives uot_sinkhorn's iterates and
 * variant 2 uot_g_sinkhorn's, within rounding. */
UOT_API size_t uot_sinkhorn_phi_workspace_size(const uot_problem* prob);
UOT_API uot_status uot_sinkhorn_phi(const uot_problem* prob, const uot_options* opt, int32_t variant, int32_t phi1,
                                    int32_t phi2, float* f, float* g, uot_result* result, void* ws, size_t ws_bytes,
                                    void* stream);

/* ---- Launch-shape tuning ------------------------------------------------------
 *
 * The launch shapes of the sweeps (rows per thread, key chunks, CTAs per SM) are
 * picked by built-in rules unless a process-wide tuning table holds a value for
 * the knob.  An entry is keyed by knob, point dimension (-1: any) and size
 * bucket floor(log2(N M)) of the sweep (-1: any); the most specific entry
 * present wins ((dim, bucket), (dim, any), (any, bucket), (any, any)).  Knobs
 * and their allowed values (every one a shape the kernels are built for):
 *   "tile.rows"          2, 4            rows per thread, tiled sweep (dim <= 3)
 *   "tile.cta_cost"      5 10 15 25 40   per-CTA fixed cost (tenths of a 128-key
 *                                        tile) in the tiled sweep's chunking
 *   "tile.waves"         1, 2, 3, 4      fewest waves of CTAs the chunking may take
 *   "points.rows"        1, 2, 4         rows per thread, direct sweep (dim <= 3)
 *   "points.resident"    2, 3, 4, 6      CTAs per SM the direct sweep's chunking aims at
 *   "dense.row_chunk"    2048 4096 8192  columns per CTA, dense row sweep
 *   "dense.col_ctas"     2, 4, 8         CTAs per SM, dense column sweep
 *   "batch.ctas_per_sm"  1, 2, 3, 4      persistent grid of uot_sinkhorn_batched
 *                                        (capped at the kernel's occupancy)
 * The entries only change launch shapes: results agree within rounding.
 * Workspaces are sized for every allowed shape, so a change of the table never
 * invalidates one (uot_workspace_size does not depend on it).  The autotuner of the
 * Python package measures the candidates on the current device and writes a
 * JSON cache, {"entries": [{"knob": K, "dim": D, "bucket": B, "value": V}, ...]};
 * uot_plan_create loads the file named by the environment variable
 * UOT_TUNE_FILE once per process.  All calls are thread-safe and touch no GPU. */

/* Sets (value != 0) or clears (value == 0) one entry.  UOT_ERR_INVALID_ARG for an
 * unknown knob, a value not allowed for it, dim outside -1..64 or bucket
 * outside -1..126. */
UOT_API uot_status uot_tune_set(const char* knob, int32_t dim, int32_t bucket, int64_t value);
/* The entry that applies to a sweep of `entries` cost entries (<= 0: bucket
 * any) in dimension dim, or 0 when the built-in rule applies. */
UOT_API uot_status uot_tune_get(const char* knob, int32_t dim, int64_t entries, int64_t* value);
/* floor(log2(entries)) (0 for entries <= 1): the size bucket of a sweep. */
UOT_API int32_t uot_tune_bucket(int64_t entries);
/* Removes every entry. */
UOT_API uot_status uot_tune_clear(void);
/* Adds the entries of a JSON tuning cache (layout above); nothing changes if
 * the file cannot be read or holds an invalid entry (UOT_ERR_INVALID_ARG). */
UOT_API uot_status uot_tune_load(const char* path);

/* Message describing the last error of the calling thread ("" if none). */
UOT_API const char* uot_last_error(void);

/* Library version string. */
UOT_API const char* uot_version(void);

#ifdef __cplusplus
}
#endif

#endif /* UOT_H */
