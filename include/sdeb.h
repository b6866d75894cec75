/*
 * sdeb.h -- C ABI of a GB300 (sm_103a) library that integrates many
 * independent orbits of an Ito SDE system with fixed-step Euler-Maruyama.
 *
 * The method is the one of SODECL (Avramidis, Lalik, Akman, arXiv 1908.03869):
 *   Eq. 1   dX_i = f_i(t, X, p) dt + sum_j g_ij(t, X, p) dW_j,
 *           n states, m Wiener processes, d parameters (Sec. 1.1);
 *   Eq. 2   X^{k+1}_i = X^k_i + f_i dt + sum_j g_ij sqrt(dt) N_j(0,1) (Sec. 2.1.1);
 *   Eq. 3   N_j from uniforms by Box-Muller, uniforms from a counter-based
 *           generator (Sec. 2.1.2);
 *   Eq. 4   output every `stride` steps (Sec. 2.1.4);
 *   Eq. 5/6 the stochastic Kuramoto model (Sec. 2.2.1);
 *   Eq. 7   the Kuramoto order parameter (Sec. 2.3.1).
 * The problem description mirrors the paper's arguments (Table 2: initial
 * states, parameter sets, orbits, n, d, m, dt, time span, steps per output).
 *
 * Conventions (every entry point):
 *   - Every call returns an sdeb_status; nothing throws across the ABI.
 *     sdeb_last_error(ctx) gives a one-line description of the last failure
 *     on that context.
 *   - A context owns all of its device buffers.  Input pointers are copied
 *     during the call (or, for device pointers, by stream-ordered copies
 *     enqueued on the given stream) and never retained.
 *   - Element type of every state / parameter / frame / gradient buffer is
 *     the context precision: float for SDEB_FP32_KAHAN, double for SDEB_FP64.
 *   - Row-major layouts: params [orbits][d] (or [d] with
 *     SDEB_FLAG_SHARED_PARAMS), states [orbits][n], frames [F][orbits][n]
 *     with F = steps / stride + 1, frame f = state at step f * stride.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Compute calls are asynchronous on that stream.
 *   - No entry point prints, aborts or falls back to the CPU.  If the CUDA
 *     runtime or the device is unavailable a call returns SDEB_ECUDA.
 *
 * Noise (reading of Sec. 2.1.2, which names Random123 but no generator or
 * layout): Philox4x32-10 (Salmon et al., SC'11) with key = (seed lo32,
 * seed hi32) and counter = (step k, noise block b = j / 4, global orbit index,
 * stream 0).  Words (w0, w1) of a block give N_{4b} (cos branch) and
 * N_{4b+1} (sin branch) with U1 = (w0 + 1/2) 2^-32 setting the radius and
 * U2 = (w1 + 1/2) 2^-32 the angle; (w2, w3) give N_{4b+2}, N_{4b+3}.  Words
 * past m are discarded.  Nothing is stored: any draw can be regenerated.
 */
#ifndef SDEB_H
#define SDEB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SDEB_API __attribute__((visibility("default")))
#else
#define SDEB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SDEB_OK = 0,
    SDEB_EINVAL = 1,        /* an argument is out of range or inconsistent */
    SDEB_ENOMEM = 2,        /* a device or host allocation failed */
    SDEB_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    SDEB_ETIMEOUT = 4,      /* a bounded device wait gave up */
    SDEB_ESTATE = 5,        /* call order violated (e.g. read before integrate) */
    SDEB_EUNSUPPORTED = 6,  /* valid request the library does not implement */
    SDEB_ENONFINITE = 7,    /* some orbit left the finite range (see sdeb_orbit_flags) */
    SDEB_EBOUNDS = 8        /* the checked build recorded an out-of-range index (sdeb_check_status) */
} sdeb_status;

/* Models (drift f and diffusion g of Eq. 1). */
enum {
    /* Kuramoto, Eq. 5/6 with one noise strength: n = m, d = n + 2,
     * p = (K, sigma, omega_1..omega_n), f_i = omega_i + K/n sum_j sin(x_j - x_i),
     * g_ij = sigma delta_ij. */
    SDEB_KURAMOTO = 1,
    /* Kuramoto in the paper's parameter layout (Eq. 5 footnote): n = m,
     * d = 2n + 1, p = (K, omega_1..omega_n, p_1..p_n), g_ij = p_i delta_ij. */
    SDEB_KURAMOTO_PAPER = 2,
    /* FitzHugh-Nagumo network of u = n/2 units, x = (v_1..v_u, w_1..w_u),
     * m = u, d = 6, p = (a, b, eps, I, c, sigma):
     * dv_i = (v_i - v_i^3/3 - w_i + I + c mean(v) - c v_i) dt + sigma v_i dW_i,
     * dw_i = eps (v_i + a - b w_i) dt. */
    SDEB_FHN_NET = 3,
    /* Ornstein-Uhlenbeck dX_i = -theta X_i dt + sigma dW_i, m = n, p = (theta, sigma). */
    SDEB_OU = 4,
    /* Geometric Brownian motion dX_i = mu X_i dt + sigma X_i dW_i, m = n, p = (mu, sigma). */
    SDEB_GBM = 5,
    /* Linear ODE (g = 0) dx_i = -theta x_i dt, m = 0, p = (theta). */
    SDEB_LINEAR_ODE = 6,
    /* A model whose drift and diffusion the caller supplies as CUDA C++
     * source, compiled at run time for this GPU (sdeb_create_user): n, m and
     * d are the caller's (1 <= n <= SDEB_USER_MAX_N, 0 <= m <= SDEB_USER_MAX_M,
     * d >= 0) and the diffusion is a dense n x m matrix. */
    SDEB_USER = 7
};

/* Precision.  FP32_KAHAN: float state with a Kahan compensation word per
 * state component, float arithmetic, FP64 time variable.  FP64: double
 * everywhere.  For the Kuramoto models under Euler-Maruyama (and Milstein)
 * the FP32 compensation is applied every 16 steps, at step multiples of
 * 16: in between, each increment enters the compensation word alone (one
 * rounding at the size of at most 16 increments), and the drift reads the
 * phase x - c.  A state kept for resuming (after sdeb_integrate_range) is the
 * pair (x, c); frames, sdeb_read_final and the allocation-free path return
 * its value x - c. */
enum { SDEB_FP32_KAHAN = 0, SDEB_FP64 = 1 };

/* Problem flags. */
enum {
    SDEB_FLAG_SHARED_PARAMS = 1u, /* one parameter vector [d] for every orbit */
    SDEB_FLAG_NO_FRAMES = 2u,     /* keep only the final state (no frame buffer) */
    /* Milstein step instead of Euler-Maruyama (the scheme the paper names as
     * the next one to add, Sec. 2.1 and Sec. 3; Kloeden and Platen's form
     * for diagonal noise): each Wiener channel j drives one state component
     * x_j with g_j(x_j), and the step adds 1/2 g_j g_j' (dW_j^2 - dt), dW_j =
     * sqrt(dt) N_j, to x_j.  This changes SDEB_GBM (g = sigma x) and the v
     * components of SDEB_FHN_NET (g = sigma v); the Kuramoto models and
     * SDEB_OU have additive noise and SDEB_LINEAR_ODE none, where Milstein
     * and Euler-Maruyama coincide.  Same noise, checkpoints and resume as
     * Euler-Maruyama.  sdeb_grad returns EUNSUPPORTED (it is the adjoint
     * of the Euler-Maruyama step). */
    SDEB_FLAG_MILSTEIN = 4u,
    /* The ODE path: classical fourth-order Runge-Kutta on the drift alone,
     * dx/dt = f(t, x, p) (the paper lists Runge-Kutta among its ODE
     * integrators, Sec. 1.5): k1 = h f(x), k2 = h f(x + k1/2), k3 = h f(x +
     * k2/2), k4 = h f(x + k3), x += (k1 + 2 k2 + 2 k3 + k4) / 6.  The
     * diffusion is not applied and no noise is drawn.  Every model, the
     * layouts sdeb_create picks (sdeb_set_layout to another layout returns
     * EUNSUPPORTED at integration).  Exclusive with SDEB_FLAG_MILSTEIN
     * (EINVAL); sdeb_grad and batches return EUNSUPPORTED. */
    SDEB_FLAG_RK4 = 8u,
    /* The ODE path, implicit Euler on the drift alone (the paper lists the
     * implicit Euler method among its ODE integrators, Sec. 1.5):
     * y = x + h f(t + h, y), solved by 4 Newton iterations from y = x, each
     * with the exact Jacobian of the built-in model's drift (a closed-form
     * solve: diagonal plus rank 2 for the Kuramoto models, which needs
     * K dt < 1; 2 x 2 blocks plus rank 1 for SDEB_FHN_NET; scalar for the
     * others).  The diffusion is not applied and no noise is drawn.  Built-in
     * models only (EUNSUPPORTED for SDEB_USER), the layouts sdeb_create picks;
     * exclusive with SDEB_FLAG_MILSTEIN, SDEB_FLAG_RK4 and
     * SDEB_FLAG_IMPLICIT_MIDPOINT (EINVAL); sdeb_grad and batches return
     * EUNSUPPORTED. */
    SDEB_FLAG_IMPLICIT_EULER = 16u,
    /* As SDEB_FLAG_IMPLICIT_EULER with the implicit midpoint rule,
     * y = x + h f(t + h/2, (x + y) / 2) (Sec. 1.5's implicit midpoint
     * method); the Kuramoto solve needs K dt < 2. */
    SDEB_FLAG_IMPLICIT_MIDPOINT = 32u
};

typedef struct {
    int32_t model;        /* SDEB_KURAMOTO ... SDEB_USER */
    int32_t n, m, d;      /* states, Wiener processes, parameters (must match the model) */
    int64_t orbits;       /* orbits in this context, >= 1 */
    double t0, dt;        /* initial time; step > 0 and finite */
    int64_t steps;        /* K >= 0, K < 2^32 */
    int64_t stride;       /* output every `stride` steps, >= 1 */
    uint64_t seed;        /* Philox key */
    int32_t precision;    /* SDEB_FP32_KAHAN or SDEB_FP64 */
    int32_t ckpt_every;   /* > 0: keep checkpoints at most ckpt_every steps apart (needed by sdeb_grad;
                             see sdeb_get_checkpoint_interval) */
    uint32_t flags;       /* SDEB_FLAG_* */
    uint32_t reserved;    /* must be 0 */
    int64_t orbit_offset; /* global index of orbit 0 (Philox keying); offset + orbits <= 2^32 */
} sdeb_problem;

typedef struct sdeb_ctx sdeb_ctx;   /* opaque, library-owned */

/* Validate the problem and allocate the context's device buffers on the
 * current CUDA device.  On failure *out is NULL and the status says why
 * (EINVAL before any CUDA call; ENOMEM / ECUDA afterwards). */
SDEB_API sdeb_status sdeb_create(const sdeb_problem *pb, sdeb_ctx **out);

/* A batch of heterogeneous problems integrated together by one persistent,
 * CUDA-graph-launched kernel (the many parameter combinations of the
 * paper's optimisation use, Sec. 1.2; the work sizing replaces the
 * hand-tuned work-group sizes of Table 4).  Each pbs[i] is validated as by
 * sdeb_create; all must be SDEB_KURAMOTO with the same precision and seed
 * and ckpt_every = 0 (EUNSUPPORTED / EINVAL otherwise), each may have its own
 * n (<= 256), orbits, t0, dt, steps, stride, flags and orbit_offset (give
 * every instance distinct global orbit indices so their noise differs).
 * Buffers are the instances' buffers concatenated in order: sdeb_set_params
 * takes params = [inst 0 params][inst 1 params]... (each [orbits_i][d_i] or
 * [d_i] if shared) and x0 = [inst 0 [orbits_i][n_i]]...; sdeb_integrate runs
 * every instance over its whole horizon (once per sdeb_set_params);
 * sdeb_batch_read reads one instance; sdeb_orbit_flags returns one byte per
 * orbit of every instance in order.  sdeb_integrate_range, sdeb_read_orbits,
 * sdeb_read_final, sdeb_grad and sdeb_set_layout return EUNSUPPORTED;
 * sdeb_autotune times candidate schedules of the whole batch. */
SDEB_API sdeb_status sdeb_create_batch(const sdeb_problem *pbs, int32_t count, sdeb_ctx **out);

/* Copy instance `instance` of a batch: what = 0 its frames
 * [steps_i/stride_i + 1][orbits_i][n_i], what = 1 its final state
 * [orbits_i][n_i]; dst_bytes exact.  ESTATE before sdeb_integrate. */
SDEB_API sdeb_status sdeb_batch_read(sdeb_ctx *ctx, int32_t instance, int32_t what, void *dst, size_t dst_bytes,
                                     int32_t dst_on_device, void *stream);

/* Schedule of a batch: queue tasks, items run as multi-warp teams (64 or
 * 128 lanes), and the persistent grid size (blocks of 128 threads). */
SDEB_API sdeb_status sdeb_batch_info(const sdeb_ctx *ctx, int32_t *tasks, int32_t *team_items, int32_t *grid);

/* Schedule knob of a batch (sdeb_autotune picks it by timing): each orbit
 * takes the layout of least total work -- 8 or 4 units per lane in a packed
 * warp, a warp of its own (2 units per lane, at most 64 units), or a
 * 64-lane (4 or 2 units per lane) or 128-lane (2) team --
 * among those whose sequential chain, steps x per-step cost, stays within
 * chain_fraction x the batch's average work per SM sub-partition, else the
 * layout with the shortest chain.  Packed warps hold several orbits side
 * by side of similar step counts.  An orbit's results depend on the
 * schedule only through its own layout (the order of its coupling sums).
 * EINVAL unless chain_fraction > 0. */
SDEB_API sdeb_status sdeb_batch_set_schedule(sdeb_ctx *ctx, double chain_fraction);

/* Layout the current schedule gives the orbits of `instance`: lanes per
 * orbit (ceil(n / units_per_lane) <= 32 in a packed warp or a warp of its
 * own, 64 or 128 for a multi-warp team) and units per lane (8, 4 or 2; 2
 * with at most 32 lanes is an orbit alone on its warp). */
SDEB_API sdeb_status sdeb_batch_layout(const sdeb_ctx *ctx, int32_t instance, int32_t *lanes, int32_t *units_per_lane);

/* Host-only view of the schedule sdeb_create_batch + sdeb_batch_set_schedule
 * (chain_fraction) would build for pbs on a device with num_sms SMs; makes no
 * CUDA call.  The problems are validated as by sdeb_create_batch.  Outputs,
 * each optional (NULL to skip):
 *   lanes, units_per_lane [count]: the layout of each instance's orbits, as
 *     sdeb_batch_layout reports it;
 *   item_task, item_slot, item_lane0 [total_orbits], one entry per orbit of
 *     every instance in order: the queue position of the orbit's task, where
 *     in the task it runs (0..3: packed warp w; 4, 5: first or second half of
 *     a two-team task; 6: the whole block) and, in a packed warp, its first
 *     lane (0 otherwise).  total_orbits must equal the sum of the instances'
 *     orbits when any of the three is given (EINVAL otherwise);
 *   ntasks: the number of queue tasks.
 * EINVAL unless chain_fraction > 0 and num_sms >= 1. */
SDEB_API sdeb_status sdeb_batch_plan(const sdeb_problem *pbs, int32_t count, double chain_fraction, int32_t num_sms,
                                     int32_t *lanes, int32_t *units_per_lane, int64_t total_orbits,
                                     int32_t *item_task, int32_t *item_slot, int32_t *item_lane0, int32_t *ntasks);

/* Limits of a user-defined model (one GPU thread integrates one orbit and
 * holds its state, drift and diffusion). */
#define SDEB_USER_MAX_N 64
#define SDEB_USER_MAX_M 64

/* A context for a user-defined model (pb->model = SDEB_USER), the GPU
 * counterpart of the paper's run-time assembly of the OpenCL kernel from
 * the user's model functions (Sec. 2.1.3, Table 1).  `source` is CUDA C++
 * (no host headers) defining, for one orbit,
 *     __device__ void sdeb_drift(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *f);
 *     __device__ void sdeb_diffusion(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *g);
 * where sdeb_real is float (SDEB_FP32_KAHAN) or double (SDEB_FP64), x[n] is
 * the state, p[d] the orbit's parameters, f[n] the drift and g[n * m] the
 * diffusion, row-major (g[i * m + j]); the macros SDEB_N, SDEB_M and SDEB_D
 * hold n, m and d.  A source that defines SDEB_DIAGONAL_NOISE (before its
 * functions) gives only g[m]: channel j drives state component j alone with
 * g_jj = g[j], the O(n) form.  The library compiles it with NVRTC for the current GPU
 * (sm_103a) together with its own step kernel: Eq. 2 with the dense
 * diffusion, X_i += f_i dt + sum_j g_ij sqrt(dt) N_j, f and g at the old
 * state and t_k = t0 + k dt, the same Philox noise and Box-Muller as the
 * built-in models, Kahan-compensated FP32 or FP64; with SDEB_FLAG_RK4 the
 * fourth-order Runge-Kutta step on the drift (sdeb_diffusion is then not
 * called but must still be defined).  One GPU thread per orbit.  The
 * context then works as one from sdeb_create (set_params, integrate,
 * integrate_range, read_orbits, read_final, orbit_flags); sdeb_set_layout,
 * sdeb_grad, SDEB_FLAG_MILSTEIN and the implicit-scheme flags return
 * EUNSUPPORTED, ckpt_every must be 0, sdeb_autotune does nothing.  EINVAL
 * with the compiler's log in sdeb_last_error(NULL) when the source does not
 * compile; EUNSUPPORTED when the run-time compiler library (libnvrtc) cannot
 * be loaded; ECUDA when the compiled kernel cannot be loaded on the device. */
SDEB_API sdeb_status sdeb_create_user(const sdeb_problem *pb, const char *source, sdeb_ctx **out);

/* Failure-detection tests inject faults on the host through the environment
 * variable SDEB_FAULT, read once per process: "alloc:<k>" makes the k-th
 * allocation of a context's buffers (counted from 0) fail, so sdeb_create
 * returns SDEB_ENOMEM; "launch:<k>" makes the k-th forward launch of an
 * integrate call (sdeb_integrate, sdeb_integrate_range; counted from 0 over
 * the process, sdeb_autotune's trial launches not counted) fail without
 * launching, so the integrate call returns SDEB_ECUDA with the step counter
 * unchanged.  Unset or any other value: no injection. */

/* Free the context and its device buffers (synchronises the device first).
 * NULL is accepted. */
SDEB_API void sdeb_destroy(sdeb_ctx *ctx);

/* Where the host-side buffer of a copy call lives (the on_device argument
 * of sdeb_set_params, the dst_on_device argument of the read calls):
 *   SDEB_MEM_HOST        host memory; the copy has completed on return;
 *   SDEB_MEM_DEVICE      device memory; the copy is ordered on `stream`;
 *   SDEB_MEM_HOST_ASYNC  host memory; the copy is only enqueued on `stream`
 *                        (it overlaps other streams' work when the buffer is
 *                        page-locked): keep the buffer alive, and unchanged
 *                        for an input, until the stream has passed the copy;
 *                        synchronise before reading an output.
 * Any other value is EINVAL. */
#define SDEB_MEM_HOST 0
#define SDEB_MEM_DEVICE 1
#define SDEB_MEM_HOST_ASYNC 2

/* Load parameter sets and initial states (Table 2 arguments "params" and
 * "initx").  params: [orbits][d] (or [d] when shared); x0: [orbits][n];
 * element type = context precision.  on_device: SDEB_MEM_* (SDEB_MEM_HOST:
 * copied before return; SDEB_MEM_DEVICE: copied on `stream`;
 * SDEB_MEM_HOST_ASYNC: host pointers copied on `stream`).  Resets the step
 * counter to 0 and writes frame 0. */
SDEB_API sdeb_status sdeb_set_params(sdeb_ctx *ctx, const void *params, const void *x0,
                            int32_t on_device, void *stream);

/* Integrate all orbits over the whole horizon k = 0..steps (Eq. 2), writing
 * frames every `stride` steps.  Requires sdeb_set_params.  Asynchronous. */
SDEB_API sdeb_status sdeb_integrate(sdeb_ctx *ctx, void *stream);

/* Integrate steps [k_begin, k_end) only; k_begin must equal the context's
 * current step (state and compensation carry over, so 0..K equals
 * 0..j + j..K bit for bit). */
SDEB_API sdeb_status sdeb_integrate_range(sdeb_ctx *ctx, int64_t k_begin, int64_t k_end, void *stream);

/* Copy frames [frame_begin, frame_begin + frame_count) into dst, layout
 * [frame_count][orbits][n]; dst_bytes must equal that size exactly.  Frames
 * past the current step are ESTATE.  dst_on_device: SDEB_MEM_*. */
SDEB_API sdeb_status sdeb_read_orbits(sdeb_ctx *ctx, void *dst, size_t dst_bytes, int64_t frame_begin,
                             int64_t frame_count, int32_t dst_on_device, void *stream);

/* Copy the current state [orbits][n] into dst (dst_bytes exact);
 * dst_on_device: SDEB_MEM_*. */
SDEB_API sdeb_status sdeb_read_final(sdeb_ctx *ctx, void *dst, size_t dst_bytes, int32_t dst_on_device,
                            void *stream);

/* Ensemble moments of the stored frames, accumulated in FP64 on the GPU
 * whatever the context precision.  The paper's accuracy experiment reports
 * the mean and the standard deviation over realisations of the order
 * parameter r(t) of Eq. 7 (Sec. 2.3); with many orbits the statistics are
 * formed where the frames are, and only these moments leave the device.
 * For the frames [frame_begin, frame_begin + frame_count):
 *   mom  [frame_count][n][2] (or NULL): per frame and state component, the
 *        mean over orbits and the population variance (divisor = orbits);
 *   rmom [frame_count][2] (or NULL): per frame, the mean over orbits and
 *        the population variance of r = |(1/n) sum_j exp(i x_j)| (Eq. 7);
 *        phase models only (SDEB_KURAMOTO, SDEB_KURAMOTO_PAPER), else
 *        EUNSUPPORTED.  r of an orbit is formed in the context precision
 *        (FP32: sine and cosine of the phase reduced to [-pi, pi] from the
 *        special-function unit), then accumulated in FP64.
 * The sums run in a fixed order -- chunks of 4096 orbits, shifted sums per
 * thread, combined by Chan, Golub and LeVeque's pairwise update in thread
 * and chunk order -- so every call gives the same bits for a frame, whatever
 * frame range it asks for.  mom_bytes / rmom_bytes must equal the sizes
 * above (ignored for a NULL pointer; at least one pointer non-NULL).
 * ESTATE for a context without frames, before sdeb_set_params, or for frames
 * past the current step; EINVAL for a range outside [0, F).  dst_on_device:
 * SDEB_MEM_* for both outputs.  Allocates its scratch stream-ordered
 * (cudaMallocAsync) and frees it on the stream.  Not for batches
 * (EUNSUPPORTED). */
SDEB_API sdeb_status sdeb_frame_moments(sdeb_ctx *ctx, int64_t frame_begin, int64_t frame_count, double *mom,
                                        size_t mom_bytes, double *rmom, size_t rmom_bytes, int32_t dst_on_device,
                                        void *stream);

/* Pathwise gradient by the discrete adjoint of Eq. 2 (checkpointed
 * recompute, Philox noise regenerated).  Requires ckpt_every > 0 and a
 * completed integration to k = steps.  All pointers are device pointers of
 * the context precision:
 *   dL_dxK [orbits][n] (input),
 *   dL_dp  [orbits][d] per orbit, or [d] summed over orbits when the
 *          parameters are shared (output),
 *   dL_dx0 [orbits][n] or NULL (output).
 * Supported models: SDEB_KURAMOTO, SDEB_KURAMOTO_PAPER (others: EUNSUPPORTED). */
SDEB_API sdeb_status sdeb_grad(sdeb_ctx *ctx, const void *dL_dxK, void *dL_dp, void *dL_dx0, void *stream);

/* Where sdeb_grad's replay keeps a segment's step records (see
 * sdeb_get_checkpoint_interval).  AUTO (the default): in shared memory when
 * the segment's records take at most 112 KB per block of 128 threads at the
 * context's layout, else in the global buffer.  GLOBAL: always the global
 * buffer.  SHARED: shared memory, and sdeb_grad returns EUNSUPPORTED where
 * they do not fit.  The two places give the same bits (the sweep takes the
 * sine and cosine of the recorded phase with the replay's own function).
 * EINVAL for another mode, a NULL or batch context. */
enum { SDEB_RECORDS_AUTO = 0, SDEB_RECORDS_GLOBAL = 1, SDEB_RECORDS_SHARED = 2 };
SDEB_API sdeb_status sdeb_set_adjoint_records(sdeb_ctx *ctx, int32_t mode);

/* Per-orbit status bits after the last integration: bit 0 = a state
 * component is not finite.  dst: host [orbits]; synchronises `stream`. */
SDEB_API sdeb_status sdeb_orbit_flags(sdeb_ctx *ctx, uint8_t *dst, void *stream);

/* Device pointer to the frame buffer ([F][orbits][n], context precision)
 * and its size, for zero-copy use; *ptr = NULL with SDEB_FLAG_NO_FRAMES.
 * The pointer stays valid until sdeb_destroy. */
SDEB_API sdeb_status sdeb_frames_device_ptr(sdeb_ctx *ctx, void **ptr, size_t *bytes);

/* Choose the lane-group layout of the context's kernels: each orbit is
 * integrated by `lanes_per_orbit` consecutive lanes (1, 2, 4, 8, 16 or 32),
 * each lane owning `units_per_lane` coupling units (a multiple of 4 when
 * lanes_per_orbit > 1).  Results depend on the layout only through the
 * order of the coupling sums, so the layout is fixed before the first
 * integration after sdeb_set_params (ESTATE otherwise) and kept for the
 * adjoint.  EINVAL if lanes x units does not cover the orbit's units,
 * EUNSUPPORTED if the model has no kernel for that layout.  sdeb_create
 * picks a default; sdeb_autotune times the candidates. */
SDEB_API sdeb_status sdeb_set_layout(sdeb_ctx *ctx, int32_t lanes_per_orbit, int32_t units_per_lane);

/* The checkpoint interval a context keeps (0 without checkpoints, and for a
 * batch).  For sdeb_grad the adjoint replays each segment between two
 * checkpoints and keeps a record of every step (each unit's sine, cosine or
 * phase, and normal; the orbit's coupling sums C, S) that its reverse sweep
 * reads back.  sdeb_create keeps checkpoints every 8 steps (when ckpt_every
 * > 8) as long as they take at most a quarter of the device memory: a
 * segment's records then fit the shared memory of the thread that writes
 * and reads them, and no record leaves the SM.  Otherwise the records go
 * through a global buffer (2 n + 2 values per orbit and step), and when
 * that buffer, for all orbits resident on the GPU at once, would outgrow
 * 60 % of the L2 cache the interval is ceil(ckpt_every / m), m <= 16,
 * rounded down to a multiple of the FP32 compensation period above it, so
 * the buffer stays on chip instead of making a round trip through HBM.
 * Checkpoint memory is (steps / interval + 1) x orbits x n elements (FP32:
 * twice that, with the compensation words).  Gradients do not depend on the
 * interval beyond rounding. */
SDEB_API sdeb_status sdeb_get_checkpoint_interval(const sdeb_ctx *ctx, int64_t *steps);
SDEB_API sdeb_status sdeb_get_layout(const sdeb_ctx *ctx, int32_t *lanes_per_orbit, int32_t *units_per_lane);

/* Layout tuner (motivated by the hand-tuned work-group sizes of the paper's
 * Table 4): times the forward kernel over the first trial_steps steps
 * (<= 0: 64) for every instantiated layout that covers the orbit's units
 * with at most 2x padding, on private copies of the current state, and keeps
 * the fastest.  A context created with ckpt_every > 0 for sdeb_grad is tuned
 * for forward + adjoint instead: both are timed over the first
 * min(ckpt_every, 1024, steps) steps (trial_steps is ignored), the adjoint
 * from checkpoint 0 with a zero dL/dX^K into temporary outputs.  Call after
 * sdeb_set_params and before integrating (ESTATE otherwise).  The context's
 * state, frames and checkpoints are untouched (the adjoint's segment scratch
 * is overwritten).  Allocates and frees temporary device buffers;
 * synchronises `stream`. */
SDEB_API sdeb_status sdeb_autotune(sdeb_ctx *ctx, int64_t trial_steps, void *stream);

SDEB_API const char *sdeb_last_error(const sdeb_ctx *ctx);
SDEB_API const char *sdeb_status_string(sdeb_status s);

/* ---- Bounds-checked build ------------------------------------------------
 * No counterpart in the paper.  The same sources compiled with SDEB_CHECKED
 * give libsdeb_checked.so (paper_1908_03869_gb300.build.build(checked=True);
 * the Python binding loads it when SDEB_LIBRARY=checked).  Its kernels
 * compare every run-time row or table index with the extent of the buffer it
 * addresses -- state rows, frame and checkpoint indices, the adjoint's
 * segment rows, a batch's task, item and instance tables and packed-warp
 * lane offsets, a user model's frame index, the moment reduction's frames --
 * and on a failed check skip the access and record (site << 48 | index) in
 * one device status word (the first failure wins).  No kernel traps.
 * sdeb_check_status synchronises the device, returns the word in *word,
 * clears it, and returns SDEB_EBOUNDS if it was set, SDEB_OK if not;
 * sdeb_check_selftest enqueues a kernel on `stream` that records site
 * 0xFFFF, index 12345 through the same path (it touches no other memory), to
 * test the reporting.  In the unchecked library both return
 * SDEB_EUNSUPPORTED without a CUDA call. */
SDEB_API sdeb_status sdeb_check_status(uint64_t *word);
SDEB_API sdeb_status sdeb_check_selftest(void *stream);

/* ---- Stand-alone kernels of the path (device pointers) ------------------ */

/* Raw Philox4x32-10 words of the Wiener stream layout: out[k][b][o][4] for
 * k in [k0, k0+nk), b in [b0, b0+nb), o in [o0, o0+no), counter stream word
 * `stream_id` (Sec. 2.1.2 reading above).  out: device uint32. */
SDEB_API sdeb_status sdeb_philox_fill(uint64_t seed, uint32_t k0, int64_t nk, uint32_t b0, int64_t nb,
                             uint32_t o0, int64_t no, uint32_t stream_id, uint32_t *out,
                             void *stream);

/* The m standard normals of Eq. 3 for steps [k0, k0+nk) and orbits
 * [o0, o0+no): out[k][o][m] in `precision` (device pointer). */
SDEB_API sdeb_status sdeb_normals_fill(uint64_t seed, uint32_t k0, int64_t nk, uint32_t o0, int64_t no,
                              int32_t m, int32_t precision, void *out, void *stream);

/* Kuramoto order parameter, Eq. 7: r[o] = |(1/n) sum_j exp(i theta[o][j])|
 * and, if dr != NULL, dr[o][l] = d r[o] / d theta[o][l] (zero where r = 0).
 * theta [orbits][n], r [orbits], dr [orbits][n]; device pointers in
 * `precision`. */
SDEB_API sdeb_status sdeb_order_param(const void *theta, int64_t orbits, int32_t n, int32_t precision,
                             void *r, void *dr, void *stream);

/* ---- Pipe rates of this GPU (the benchmark's roofline peaks) ------------
 * No counterpart in the paper.  Measures the issue rate of one arithmetic
 * pipe in results per SM per clock: pipe 0 = SFU sine (sin.approx.ftz.f32),
 * 1 = SFU base-2 logarithm, 2 = SFU square root (sqrt.approx.ftz.f32),
 * 3 = FP64 fused multiply-add, 4 = FP32 fused multiply-add.  One block of
 * 1024 threads per SM runs 8 independent chains of `iters` (1 .. 2^24)
 * dependent operations per thread; the median over the SMs of the block's
 * clock64 cycles divides its 8192 * iters operations.  The rate per clock is
 * independent of the clock frequency.  Synchronises `stream`; allocates
 * stream-ordered scratch.  EINVAL on a bad argument, ECUDA on a failure. */
SDEB_API sdeb_status sdeb_pipe_rate(int32_t pipe, int32_t iters, double *ops_per_clk_per_sm, void *stream);

/* ---- Allocation-free forward integration ------------------------------
 * No counterpart in the paper.  For callers that cannot allocate device
 * memory -- code running while a CUDA graph is captured, hosts whose own
 * allocator owns every device byte, embedded or real-time programs that
 * forbid allocation after start-up -- sdeb_create is unusable because the
 * context allocates its buffers.  This entry point allocates nothing: the
 * caller passes the inputs and outputs, and the only scratch (the FP32 Kahan
 * compensation words and a per-orbit status byte) lives in a fixed array
 * compiled into the library, SDEB_NOALLOC_SCRATCH_BYTES bytes that every GPU
 * which loads the library keeps until the process exits.
 *
 * Semantics are those of sdeb_create + sdeb_set_params(on_device = 1) +
 * sdeb_integrate + reading the frames and the final state, for the same
 * problem, with the context at the layout sdeb_create picks: the same kernel
 * at the same layout produces the same bits.  (A context retuned by
 * sdeb_autotune or sdeb_set_layout sums the coupling terms in another order
 * and agrees within the FP32 / FP64 parity tolerances, not bit for bit.)
 *   pb       problem; ckpt_every must be 0; orbits <= SDEB_NOALLOC_MAX_ORBITS
 *            and orbits * n <= SDEB_NOALLOC_MAX_STATES, else SDEB_EINVAL.
 *   params   device, [orbits][d] (or [d] with SDEB_FLAG_SHARED_PARAMS).
 *   x0       device, [orbits][n], not modified.
 *   x_final  device, [orbits][n]; receives x0, then serves as the working
 *            state and ends as the state at step `steps`.
 *   frames   device, [steps/stride + 1][orbits][n], or NULL for no frames.
 * Element type is the problem precision.  Asynchronous on `stream`.
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current) and remembers it with the
 * identity of the CUDA context; a call in a different context of the device
 * (after cudaDeviceReset, or the primary context released and re-created)
 * looks it up again.  Make a call that looks up -- the first one on a device,
 * and the first after its context changed -- before any stream capture.  Calls share the scratch and it keeps the last
 * call's contents (each call clears what must start at zero): calls whose
 * work overlaps on the GPU race, so serialise them (one stream, or events).
 * Non-finite orbits are not reported on this path. */
#define SDEB_NOALLOC_MAX_STATES (1 << 21)
#define SDEB_NOALLOC_MAX_ORBITS (1 << 21)
#define SDEB_NOALLOC_SCRATCH_BYTES (SDEB_NOALLOC_MAX_STATES * 4 + SDEB_NOALLOC_MAX_ORBITS)
SDEB_API sdeb_status sdeb_integrate_noalloc(const sdeb_problem *pb, const void *params, const void *x0,
                                            void *x_final, void *frames, void *stream);

/* ---- Particle swarm search over model parameters ------------------------
 * The population-based parameter optimisation the paper builds the
 * integrator for (Sec. 1.2: an EA or a particle swarm integrates the model
 * over every parameter set of its population each generation, with several
 * realisations per set against the noise).  A generation is
 *   sdeb_swarm_expand   particles -> per-orbit parameter rows,
 *   sdeb_set_params(on_device = 1) + sdeb_integrate   (or the noalloc path),
 *   sdeb_swarm_fitness  final states -> one fitness per particle,
 *   sdeb_swarm_update   personal and global bests, velocities, positions,
 * all asynchronous on one stream, nothing read back in between.  P particles
 * of D <= SDEB_SWARM_MAX_DIMS dimensions; particle i's realisation q is
 * orbit i R + q.  Swarm arrays are FP64 device arrays, row-major:
 * x, v, pbest [P][D], pbest_fit, fit [P].  Host arrays (dims, lo, hi) are
 * read during the call.  EINVAL on NULL pointers, P < 1, R < 1, D outside
 * [1, SDEB_SWARM_MAX_DIMS], a column outside [0, d), lo > hi; ECUDA on a
 * launch error. */
#define SDEB_SWARM_MAX_DIMS 16

/* params_out[i R + q][c] = x[i][j] where c == dims[j], else base[c]:
 * base [d] and params_out [P R][d] device, in `precision` (x rounded to
 * FP32 for SDEB_FP32_KAHAN); dims [D] host, distinct columns. */
SDEB_API sdeb_status sdeb_swarm_expand(const double *x, int64_t particles, int32_t dims_count,
                                       const int32_t *dims, const void *base, int32_t d, int32_t realisations,
                                       int32_t precision, void *params_out, void *stream);

/* fit[i] = (mean over q of r(theta[i R + q]) - r_target)^2 with r the order
 * parameter of Eq. 7, computed in FP64 from theta [P R][n] (device, in
 * `precision`); the realisations are summed in a fixed order. */
SDEB_API sdeb_status sdeb_swarm_fitness(const void *theta, int64_t particles, int32_t realisations, int32_t n,
                                        int32_t precision, double r_target, double *fit, void *stream);

/* One generation g of the inertia-weight particle swarm (Kennedy and
 * Eberhart; inertia weight of Shi and Eberhart), minimising the fitness:
 *   where fit[i] < pbest_fit[i]: pbest[i] = x[i], pbest_fit[i] = fit[i]
 *     (a NaN fitness never improves; start pbest_fit at +inf);
 *   b = the least pbest_fit, the lowest index among equals -> *gbest;
 *   v = w v + c1 r1 (pbest[i] - x[i]) + c2 r2 (pbest[b] - x[i]), clamped
 *   to +-(hi - lo); x = x + v clamped to [lo, hi], per dimension;
 * r1, r2 = (w + 1/2) 2^-32 of words 0 and 1 of Philox4x32-10 with key `seed`
 * and counter (g, j, i, 2) -- the noise generator on counter stream 2.  Each
 * product and sum is rounded separately, in the order written.  x, v, pbest,
 * pbest_fit updated in place; fit [P] and gbest (one int32) device; lo, hi
 * [D] host.  P <= 2^24. */
SDEB_API sdeb_status sdeb_swarm_update(double *x, double *v, double *pbest, double *pbest_fit, const double *fit,
                                       int64_t particles, int32_t dims_count, const double *lo, const double *hi,
                                       double w, double c1, double c2, uint64_t seed, uint32_t generation,
                                       int32_t *gbest, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SDEB_H */
