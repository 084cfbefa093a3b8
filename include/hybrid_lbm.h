/*
 * hybrid_lbm.h -- C ABI of the GB300 (sm_103a) implementation of the hybrid
 * free-energy lattice Boltzmann scheme for binary fluid mixtures of
 * Tiribocchi, Stella, Gonnella and Lamura (arXiv:0902.3921).
 *
 * One LB step (Sec. II) is, at every lattice site r of a periodic
 * Lx x Ly (x Lz) lattice with unit spacing and unit LB time step:
 *   1. mu = a phi + b phi^3 - kappa lap_D phi                         (Eq. 5)
 *   2. F  = -phi d_D mu [+ d_D((cs^2 - T) n)] [+ n g while t < force_steps]
 *                                                              (Eq. 28, Sec. III)
 *      with the 3x3 "stencil" operators d_D (N, M) and lap_D (Q, R) of
 *      Eqs. 30-31 (M = (1-2N)/4, R = (1-Q)/2; D3Q19: M = (1-2N)/8, R = (1-Q)/4)
 *   3. n = sum_i f_i, n u* = sum_i f_i e_i + F/2                  (Eqs. 12, 18)
 *   4. f_i(r + e_i, t+1) = f_i - (f_i - feq_i(n, u*))/tau + F_i
 *      with feq of Eq. 15 and the forcing term F_i of Eq. 29       (Eq. 17)
 *   5. phi(t) -> phi(t+1) by m substeps of dt = 1/m (Sec. II C), each an
 *      upwind convective half step (Eqs. 32-35) with u*(t) and an explicit
 *      diffusive half step (Eq. 36) with the 5-point (7-point) Laplacian.
 * Both halves of a step read the state at time t.  Lattices: D2Q9 (Sec. II A,
 * Fig. 1) and its 3D generalisation D3Q19.
 *
 * Conventions for every entry point:
 *   - Host arrays are caller-owned, read or written only during the call,
 *     row-major [z][y][x] (site s = (z*Ly + y)*Lx + x), FP64.
 *   - The handle owns all device memory it allocates.  Calls on one handle
 *     are not thread-safe; distinct handles are independent.
 *   - Work is queued on the handle's CUDA stream.  lbm_step returns without
 *     waiting; every other call that returns data waits for the stream.
 *   - Errors are negative return codes, latched on the handle: after an
 *     error the handle refuses further work (except lbm_free and
 *     lbm_last_error) and lbm_last_error() says what failed.  Nothing aborts
 *     the process.
 */
#ifndef HYBRID_LBM_H
#define HYBRID_LBM_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LBM_OK = 0,
  LBM_EINVAL = -1,     /* bad parameter, size or pointer                      */
  LBM_ECUDA = -2,      /* a CUDA runtime call failed                          */
  LBM_ENOMEM = -3,     /* device allocation failed                            */
  LBM_ENONFINITE = -4, /* NaN or Inf found by lbm_diagnostics                 */
  LBM_ETIMEOUT = -5,   /* a bounded device wait gave up                       */
  LBM_ESTATE = -6      /* call out of order (e.g. lbm_step before init)      */
};

/* Storage/compute precision of the populations (h_i = f_i - w_i is stored). */
enum {
  LBM_F64 = 0,    /* FP64 populations, phi and arithmetic                      */
  LBM_F32DEV = 1, /* FP32 deviations h_i = f_i - w_i, FP32 phi and arithmetic  */
  LBM_F16DEV = 2  /* FP16 deviations scaled by 2^f16_scale_log2, FP32 phi and
                     arithmetic                                                */
};

enum {
  LBM_ADV_PAPER = 0, /* Eqs. 32-35 as printed (does not conserve sum phi)     */
  LBM_ADV_FLUX = 1   /* conservative upwind flux form, same stencil radius    */
};

typedef struct {
  int dims;              /* 2 (D2Q9) or 3 (D3Q19)                              */
  int Lx, Ly, Lz;        /* periodic lattice, each >= 3; Lz ignored in 2D      */
  double a, b, kappa;    /* free energy, Eq. 1; b > 0, kappa >= 0              */
  double T;              /* temperature of the ideal-gas term (Eqs. 1, 28)     */
  double tau;            /* relaxation time (Eq. 11), > 1/2                    */
  double Gamma;          /* mobility (Eq. 10), >= 0                            */
  double N, Q;           /* stencil parameters of Eqs. 30-31                   */
  int fd_substeps;       /* m of Sec. II C: 0 = smallest m with the diffusive
                            step's stiffness * dt <= 1.5; m > 0 must meet the
                            Euler bound (stiffness * dt <= 2); m < 0 forces |m| */
  int adv_variant;       /* LBM_ADV_PAPER or LBM_ADV_FLUX                       */
  int cubic_at_half;     /* 0: b lap (phi^n)^3 as in Eq. 36; 1: cube of phi^{n+1/2} */
  double g[3];           /* body force per unit density, G = n g (Sec. III)    */
  long long force_steps; /* G acts at steps t = 0 .. force_steps-1             */
  int precision;         /* LBM_F64, LBM_F32DEV or LBM_F16DEV                  */
  int f16_scale_log2;    /* FP16 scale exponent s (0 = default 10), 0..14      */
  int stencil_fd;        /* 0: Eqs. 33 and 36 as printed (central d u, 5-point
                            Laplacian); 1: the stencil operators of Eqs. 30-31
                            at this N, Q for d u and the three Laplacians of
                            Eq. 36 -- the "more general stencil" of Sec. II C
                            (after Eq. 36) and Sec. IV.  2D, the printed
                            advection form and Q >= 0 only (EINVAL otherwise);
                            run by the shared-memory tile FD kernel.  lap_D's
                            largest eigenvalue is max(8Q, 4) (8 for the
                            5-point form), which the m of fd_substeps = 0 and
                            the Euler bound take into account               */
} lbm_params;

/* FP64 observables (Sec. III) at the handle's current time t. */
typedef struct {
  long long t;
  double sum_n;       /* sum of n over all sites                               */
  double sum_phi;     /* sum of phi                                            */
  double momentum[3]; /* sum of n u*                                           */
  double u_max;       /* max |u*| (Table I reports u_max / c_s)                */
  double dp;          /* p0(centre site) - p0(site 0), p0 of Eq. 6 with the
                         stencil operators: the Laplace jump of a centred drop */
  double r_cm[3];     /* sum phi r / sum phi over sites with phi > 0 (Eq. 40),
                         periodic images nearest to the previous r_cm (the box
                         centre before the first call)                         */
  double v_f[3];      /* u* at r_cm, bi/trilinear, periodic (Sec. III)          */
  double area;        /* sum (1 + phi/phi0)/2, phi0 = sqrt(-a/b) (or 1 if a>=0)*/
  double R_eff;       /* sqrt(area/pi) in 2D, (3 area / 4 pi)^(1/3) in 3D      */
  int nonfinite;      /* 1 if any n, u* or phi is NaN or Inf                   */
} lbm_diag;

typedef struct lbm_handle lbm_handle;

/* Validates *params (EINVAL: tau <= 1/2, b <= 0, kappa < 0, Gamma < 0, a side
 * < 3, dims not 2 or 3, N or Q not finite, a requested m below the Euler bound,
 * unknown precision/variant), picks m (Sec. II C), allocates device memory and
 * returns a handle in *out (NULL on error; the error text is then available
 * from lbm_last_error(NULL)).  cuda_stream is a cudaStream_t to queue work on,
 * or NULL for a stream owned by the handle.  Does not initialise the fields.
 * Testing the error paths (environment, read at each call):
 *   LBM_FAULT=alloc    lbm_create returns LBM_ENOMEM as if the first device
 *                      allocation failed, before any CUDA call;
 *   LBM_FAULT=alloc:K  the K-th device allocation fails (LBM_ENOMEM; the
 *                      earlier ones are freed);
 *   LBM_FAULT=h2d      lbm_init_fields fails as if its host-to-device copy
 *                      had (LBM_ECUDA, latched on the handle);
 *   HLBM_DEBUG_TMA_WAIT_NS=<ns>  bound of the TMA collide kernels' waits for
 *                      a tile's copies, and of the opt-in one-kernel 3D FD
 *                      substep's waits for its staged u and v rows (default
 *                      0.5 s; process-wide, set by each lbm_create).  A short
 *                      bound makes the wait give up: the kernel lets its
 *                      issued copies land (that drain keeps the 0.5 s
 *                      bound), skips its work, and the handle reports
 *                      LBM_ETIMEOUT at the next lbm_moments,
 *                      lbm_diagnostics or lbm_synchronize.  The handle can
 *                      then only be freed.
 *   HLBM_FD3_FUSED_ADV=1  3D, FP32, Lx = 128 or 256: each FD substep as one
 *                      software-pipelined kernel (advection, psi and the new
 *                      phi; the same results as the default two kernels,
 *                      slower on the GB300).
 * Launch choices (environment, read at creation or once per process):
 *   HLBM_TUNING=sub,rows,cols,collide_rows[,tile]  fixed 2D launch shapes
 *                      instead of the autotuner's timed choice (lbm_tuning
 *                      reports either); HLBM_TUNE_VERBOSE=1 prints the timings;
 *   HLBM_PDL=1         programmatic dependent launches between the step's
 *                      kernels (off by default: slower on the GB300). */
int lbm_create(const lbm_params *params, void *cuda_stream, lbm_handle **out);

/* Device buffers a caller (for example a PyTorch program) allocates and lends
 * to a handle: the two population lattices (q planes of S sites each, q = 9
 * or 19, element type FP64 / FP32 / FP16 as the precision stores deviations),
 * the three phi planes (t, t+1, FD scratch) and the dims velocity planes u*
 * (FP64 in LBM_F64, FP32 otherwise).  Each pointer must be 16-byte aligned
 * and hold at least the byte count lbm_buffer_bytes reports. */
typedef struct {
  void *populations[2];
  void *phi[3];
  void *u;
} lbm_buffers;

/* Byte counts of the lbm_buffers members for *params: bytes[0] for each
 * population lattice, bytes[1] for each phi plane, bytes[2] for u*.  Pure
 * arithmetic (no CUDA call); EINVAL as lbm_create's validation. */
int lbm_buffer_bytes(const lbm_params *params, unsigned long long bytes[3]);

/* lbm_create on caller-owned buffers (the handle adopts them):
 * the handle reads and writes them but never frees them; they must outlive
 * the handle.  Everything else (FP64 staging, diagnostics scratch, the 3D FD
 * planes) is still allocated by the handle.  EINVAL for a NULL or unaligned
 * buffer, before any CUDA call. */
int lbm_create_with_buffers(const lbm_params *params, void *cuda_stream, const lbm_buffers *buffers,
                            lbm_handle **out);

/* Sets t = 0, phi(0) = phi and populations f_i = feq_i(n, u - F/(2n)) (Eqs. 15,
 * 18), F from Eq. 28 at t = 0, so that the u* of Eq. 18 at t = 0 equals u.
 * n, phi, ux, uy (and uz in 3D; ignored and may be NULL in 2D) are host arrays
 * of Lx*Ly*Lz doubles.  n must be > 0 (not checked per site). */
int lbm_init_fields(lbm_handle *h, const double *n, const double *phi,
                    const double *ux, const double *uy, const double *uz);

/* Advances nsteps >= 0 LB steps (each: one LB step and m FD substeps).
 * Asynchronous: returns once the work is queued (CUDA graphs when enabled).
 * ESTATE before lbm_init_fields/lbm_load. */
int lbm_step(lbm_handle *h, long long nsteps);

/* n(t), phi(t) and u*(t) (Eq. 18, including F/2) into host arrays of Lx*Ly*Lz
 * doubles; any output pointer may be NULL to skip it.  Waits for the stream. */
int lbm_moments(lbm_handle *h, double *n, double *phi, double *ux, double *uy,
                double *uz);

/* The pre-collision populations f_i(r, t) as a host array [q][z][y][x] of
 * doubles, q = 9 (D2Q9) or 19 (D3Q19), in the direction order of lbm_lattice. */
int lbm_populations(lbm_handle *h, double *f);

/* Copies the lattice vectors (q rows of 3 ints) and weights (q doubles) used by
 * lbm_populations; either pointer may be NULL.  Returns q, or EINVAL. */
int lbm_lattice(int dims, int *e, double *w);

/* FP64 diagnostics at the current t (deterministic reduction order).  Returns
 * ENONFINITE (and fills *out) when a NaN/Inf is found; the handle stays usable. */
int lbm_diagnostics(lbm_handle *h, lbm_diag *out);

/* Waits for all queued work; returns the first latched error. */
int lbm_synchronize(lbm_handle *h);

long long lbm_time(const lbm_handle *h);       /* current LB step t, or -1     */

/* The launch shapes picked by the autotuner of lbm_create (2D; it times the
 * candidates with CUDA events on the handle's own buffers): writes up to n of
 * {FD substeps per launch, FD output rows per warp (block kernel: region
 * rows), FD columns per lane (block kernel: warps / 8), collide kernel (0 / 1:
 * cp.async staging sized for 4 / 3 CTAs per SM; 2 / 4: sites per thread of
 * the register kernel; 3, 5, 6: TMA staging with the scalar collision or the
 * packed-pair collision for 4 / 3 CTAs per SM, FP32 and FP16 storage; 7:
 * persistent pipelined TMA kernel, FP32), m, FD kernel (0: warp-marching;
 * 32 or 64: shared-memory tile of that width; 128: block kernel; 1:
 * y-marching wavefront kernel, whose "rows" are the output rows of one
 * segment and whose substeps per launch are 2 or 4)} into values
 * and returns 6 (EINVAL on NULL).
 * Environment: HLBM_TUNING="sub,rows,cols,collide_rows[,tile]" fixes the shapes
 * instead of timing them (reproducible profiling); HLBM_TUNE_VERBOSE=1 prints
 * every candidate's time to stderr. */
int lbm_tuning(const lbm_handle *h, int *values, int n);
int lbm_fd_substeps(const lbm_handle *h);      /* the m in use, or -1          */

/* 1 (default) captures lbm_step into CUDA graphs; 0 launches kernels one by
 * one.  Kernel timing (below) forces one-by-one launches. */
int lbm_set_graphs(lbm_handle *h, int enable);

/* When enabled, every kernel of lbm_step is bracketed by CUDA events on the
 * handle's stream and lbm_kernel_times returns, per kernel family, the summed
 * milliseconds and launch counts since the last reset.  Families:
 * 0 = collide/stream (steps 1-4), 1 = FD update (step 5), 2 = density (only
 * when T != 1/3).  ms and launches point to arrays of 3; reset != 0 clears. */
int lbm_set_kernel_timing(lbm_handle *h, int enable);
int lbm_kernel_times(lbm_handle *h, double *ms, long long *launches, int reset);

/* Raw checkpoint: header (magic, version, parameters, t, precision, CRC32)
 * followed by the device state.  lbm_load needs a handle created with equal
 * parameters and restores t.  A file it cannot use (unreadable, another
 * format or version, other parameters, truncated, CRC mismatch) returns
 * EINVAL without latching: the handle stays usable and lbm_last_error names
 * the reason. */
int lbm_save(lbm_handle *h, const char *path);
int lbm_load(lbm_handle *h, const char *path);

/* ---- batches of independent lattices --------------------------------------
 * Many independent periodic 2D (D2Q9) lattices of uneven size, all with the
 * common parameters of `common` (T = 1/3, FP64 or FP32-deviation storage)
 * and each with its own size and body force G = n g while t < force_steps
 * (Sec. III), advanced together by one of two paths chosen at creation:
 *   persistent: ONE kernel launch per lbm_batch_step call, each instance
 *     owned by one CTA, so no CTA ever waits for another; its CTA shape
 *     (threads x CTAs per SM) is timed on a zeroed state and the fastest kept
 *     (HLBM_BATCH_SHAPE="threads,ctas_per_sm" fixes it);
 *   tiled (FP32 deviations, printed advection form, even m, every Lx a
 *     multiple of 4): per LB step the collide over the 32 x 16 tiles of all
 *     instances -- a persistent TMA-staged kernel, through one set of tensor
 *     maps per instance shape, for the instances at least 64 on a side
 *     (HLBM_BATCH_NO_TMA=1 sends them to the tile kernel too), the tile
 *     kernel for the rest -- and m / 2 launches of the two-substep wavefront
 *     FD kernel over their 128-column strips, in segments of at most 48 rows
 *     (HLBM_BATCH_FD_ROWS=n changes the 48).
 * Where the tiled path is eligible both are timed and the faster kept
 * (HLBM_BATCH_PATH=tiled|persistent fixes the choice; HLBM_TUNE_VERBOSE=1
 * prints the timings).  Either is captured in a CUDA graph per call.  Every
 * instance starts at rest (phi = 0, n = 1, u = 0).  Instances are stored
 * grouped by shape; the instance index k of the calls below is the index in
 * the array given to lbm_batch_create. */
typedef struct {
  int Lx, Ly;            /* periodic lattice of this instance, each >= 3        */
  double g[2];           /* body force per unit density                         */
  long long force_steps; /* g acts at steps t = 0 .. force_steps-1             */
} lbm_instance;

typedef struct lbm_batch lbm_batch;

/* Validates and allocates; returns the batch in *out (NULL and the error text
 * in lbm_batch_last_error(NULL) on failure).  cuda_stream as in lbm_create. */
int lbm_batch_create(const lbm_params *common, const lbm_instance *inst, int count,
                     void *cuda_stream, lbm_batch **out);
/* Initial fields of instance k (host FP64 arrays of Lx*Ly values), as in
 * lbm_init_fields.  Resets the batch clock to t = 0: initialise every instance
 * that should not start at rest before the first lbm_batch_step. */
int lbm_batch_init_fields(lbm_batch *b, int k, const double *n, const double *phi,
                          const double *ux, const double *uy);
/* Advances every instance by nsteps LB steps on the chosen path.  On the
 * tiled path, a TMA copy that never completes ends the collide after its
 * bounded wait and latches LBM_ETIMEOUT at the next lbm_batch_synchronize or
 * lbm_batch_moments. */
int lbm_batch_step(lbm_batch *b, long long nsteps);
/* n, phi, u* of instance k at the current t into host arrays (NULL skips). */
int lbm_batch_moments(lbm_batch *b, int k, double *n, double *phi, double *ux, double *uy);
int lbm_batch_set_graphs(lbm_batch *b, int enable);
/* Threads per CTA, CTAs and total sites of the batch (any pointer may be
 * NULL); the tiled path reports 0 threads and its number of collide tiles. */
int lbm_batch_shape(const lbm_batch *b, int *threads, int *ctas, long long *sites);
int lbm_batch_synchronize(lbm_batch *b);
void lbm_batch_free(lbm_batch *b);
const char *lbm_batch_last_error(const lbm_batch *b);

/* ---- learned surrogate ------------------------------------------------------
 * A stack of periodic 3x3 convolutions (4 -> C -> ... -> C -> 4 channels, ReLU
 * between layers) that predicts, from the state x_t = (phi, u*_x, u*_y, n - 1)
 * of a 2D lattice, the state one window of k LB steps later:
 *   x_{t+k} = x_t + out_std * Net((x_t - in_mean) / in_std).
 * BF16 weights and activations, FP32 accumulation on the tensor cores, FP32
 * master weights and Adam.  The paper has no counterpart: this is the learned
 * extension of the method, judged by the paper's observables (structure
 * factor, domain size, mass).  States are device FP32 arrays [N][H][W][4];
 * H must be a multiple of 8 and W of 16. */
typedef struct lbm_net lbm_net;

/* channels 16 or 32, layers 2..8; He-normal weights from `seed`, zero biases. */
int lbm_net_create(int channels, int layers, unsigned long long seed, lbm_net **out);
/* Number of parameters in the flat order [layer][W[co][3][3][ci] then b[co]]. */
long long lbm_net_param_count(const lbm_net *net);
/* Copies the FP32 master parameters to (set = 0) or from (set = 1) a host
 * array of lbm_net_param_count floats. */
int lbm_net_params(lbm_net *net, float *host, long long n, int set);
/* The gradients of the last lbm_net_train_step, same order. */
int lbm_net_grads(lbm_net *net, float *host, long long n);
/* Per-channel normalisation: in_mean[4], in_std[4] of x_t and out_std[4] of
 * x_{t+k} - x_t (host arrays). */
int lbm_net_set_normalisation(lbm_net *net, const float *in_mean, const float *in_std,
                              const float *out_std);
int lbm_net_normalisation(const lbm_net *net, float *out12);
/* x1 = prediction of the state one window after x0 (device arrays). */
int lbm_net_forward(lbm_net *net, const float *x0, int N, int H, int W, float *x1,
                    void *cuda_stream);
/* Timing of the forward pass: runs it reps + 1 times on x0 (device array,
 * first run a warm-up) with CUDA events recorded on the stream around each
 * convolution launch, and writes the mean milliseconds of each layer's launch
 * into the host array ms[layers]; synchronises the stream.  The paper has no
 * counterpart (a measurement entry point). */
int lbm_net_layer_times(lbm_net *net, const float *x0, int N, int H, int W, int reps, float *ms,
                        void *cuda_stream);
/* One training step on pairs (x0, x1): MSE between Net(x0) and the normalised
 * change, backward pass, and (update != 0) one Adam step with rate lr.  *loss
 * (may be NULL) receives the loss before the update; waits for the stream. */
int lbm_net_train_step(lbm_net *net, const float *x0, const float *x1, int N, int H, int W,
                       float lr, int update, double *loss, void *cuda_stream);
/* The network state of lattice h at its current time into a device array
 * [Ly][Lx][4] (queued on h's stream). */
int lbm_surrogate_state(lbm_handle *h, float *out);
/* Advances h by `windows` windows of `window_steps` LB steps each with the
 * network: state -> prediction -> residual check (mean change of phi per site
 * |d sum phi| / sites <= mass_tol; max |phi| <= min(max(1.1 phi0, 1.05
 * max|phi_t|), 1.5 phi0); max |u*| <= min(max(1.5 max|u*_t|, 0.01 c_s),
 * 0.5 c_s); max |n - 1| <= min(max(2 max|n_t - 1|, 1e-3), 0.3); every value
 * finite; with _t the state the window starts from; the ceilings keep
 * accepted windows from compounding the relative bounds;
 * HLBM_SURROGATE_VERBOSE=1 prints the values per window); a passing
 * prediction becomes the new state (populations rebuilt as f_eq(n, u* - F/2n)
 * with phi shifted to keep sum phi if conserve_mass), a failing one is
 * replaced by window_steps plain LB steps.  phi_clamp > 0 first clips the
 * predicted phi to |phi| <= phi_clamp * max|phi_t|.  *fallbacks counts the
 * plain windows.  The body force must be off; t advances by
 * windows * window_steps. */
int lbm_surrogate_advance(lbm_handle *h, lbm_net *net, int windows, int window_steps,
                          double mass_tol, int conserve_mass, double phi_clamp, int *fallbacks);
/* As lbm_surrogate_advance, with relax_steps >= 0 plain LB steps after every
 * prediction: the predicted state becomes the lattice state, relax_steps
 * steps run, and the residual check applies to the relaxed state; a failing
 * window restores the populations and phi of its start (kept in a device
 * copy owned by net) and runs window_steps + relax_steps plain steps.  Each
 * window advances t by window_steps + relax_steps; relax_steps = 0 is
 * lbm_surrogate_advance. */
int lbm_surrogate_advance_relaxed(lbm_handle *h, lbm_net *net, int windows, int window_steps,
                                  int relax_steps, double mass_tol, int conserve_mass, double phi_clamp,
                                  int *fallbacks);
void lbm_net_free(lbm_net *net);
const char *lbm_net_last_error(const lbm_net *net);

/* Allocation-free diagnostics.  The paper has no counterpart to this entry
 * point: it exists for callers that cannot allocate device memory, such as a
 * host framework that owns all device memory through its own allocator and
 * budget, or a time-critical loop in which cudaMalloc/cudaFree would
 * synchronise the device.  It computes the same FP64 observables as
 * lbm_diagnostics, with the same kernels, from fields the caller passes in,
 * and allocates nothing: its scratch (per-block partial sums and the result
 * vector, LBM_NOALLOC_MAX_BLOCKS * 12 + 19 doubles, about 192 KiB) is a
 * static device array that every GPU using the library holds until the
 * process exits.
 *
 *   params  geometry and the a, b, kappa, T, N, Q used by p0; other fields
 *           are ignored.  They are checked as lbm_create checks them (sides
 *           >= 3; a finite and < 0, so that phi0 = sqrt(-a/b); b > 0; kappa
 *           >= 0; T > 0; N and Q finite), and at most LBM_NOALLOC_MAX_SITES
 *           sites: anything else returns LBM_EINVAL with a reason before
 *           any CUDA call ("exceed the ... capacity" for a lattice too big).
 *   fields  DEVICE pointer to (2 + dims) * S doubles, [n | phi | u*_x | u*_y
 *           (| u*_z)], each block row-major [z][y][x] (what lbm_moments
 *           returns, laid end to end).  Read only.
 *   r_ref   host array of 3 doubles: the reference point of the periodic
 *           centre-of-mass unwrap (lbm_diagnostics uses the previous r_cm),
 *           or NULL for the box centre.
 *   cuda_stream  the stream to run on (NULL: the legacy default stream).
 *   out     host struct, filled on return (out->t = -1).
 * Waits for the stream.  Returns LBM_OK, LBM_ENONFINITE (out filled),
 * LBM_EINVAL or LBM_ECUDA; lbm_noalloc_last_error() describes the failure.
 * The first call in each CUDA context looks up the device address of the
 * scratch array with that context current (the address belongs to the
 * context: after cudaDeviceReset, or under another context of the same
 * device, the next call looks it up again); make that first call in a
 * context before any stream capture.  All calls share the one array and leave the last call's values
 * in it (each call writes every entry it reads, so nothing is cleared):
 * calls that overlap on the GPU (other streams, other host threads) race. */
#define LBM_NOALLOC_MAX_BLOCKS 2048
#define LBM_NOALLOC_MAX_SITES (LBM_NOALLOC_MAX_BLOCKS * 2048)
int lbm_diagnostics_noalloc(const lbm_params *params, const double *fields,
                            const double *r_ref, void *cuda_stream, lbm_diag *out);
const char *lbm_noalloc_last_error(void);

/* Frees the handle and its device memory (and its stream if it owns one).
 * NULL-safe.  Does not free a caller-provided stream. */
void lbm_free(lbm_handle *h);

/* Text of the last error on h (or of the last failed lbm_create if h is
 * NULL); "" when there is none.  Valid until the next call on h. */
const char *lbm_last_error(const lbm_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* HYBRID_LBM_H */
