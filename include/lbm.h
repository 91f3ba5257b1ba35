/*
 * lbm.h -- C ABI of the GB300 lattice Boltzmann outflow library.
 *
 * The library advances a 2D D2Q9 lattice Boltzmann simulation on one GPU:
 * a fused pull-stream-and-collide step (BGK or MRT) with full-way bounce-back
 * walls and momentum-exchange forces, a Zou & He velocity inlet on the west
 * edge, and an east outflow that rebuilds the unknown incoming populations
 * f3, f6, f7 by Zou & He, by a small neural network, or by a characteristic
 * boundary condition.  This follows "Reduction of Outflow Boundary Influence
 * on Aerodynamic Performance using Neural Networks" (arXiv 2506.05293),
 * cited below by section and equation.
 *
 * Conventions for every entry point:
 *  - Every call returns an lbm_status; nothing throws across the ABI.  On an
 *    error lbm_last_error() gives a message (thread-local, valid until the
 *    next call on that thread).
 *  - Host arrays passed in are copied before the call returns; the caller
 *    keeps ownership.  Host arrays passed out are written in full.
 *  - 2D host arrays are row-major (ny rows of nx values, x fastest);
 *    population arrays are (9, ny, nx) with the direction slowest.
 *  - Velocities: c0=(0,0) c1=(1,0) c2=(0,1) c3=(-1,0) c4=(0,-1) c5=(1,1)
 *    c6=(-1,1) c7=(-1,-1) c8=(1,-1); weights 4/9, 1/9 (1-4), 1/36 (5-8).
 *  - Work is enqueued on the simulation's CUDA stream.  lbm_step never
 *    blocks; calls that return data to the host synchronise that stream.
 *    Device-side faults (non-finite density) are latched in a status word
 *    that lbm_sync and the data-returning calls report.
 *  - Calls on one lbm_sim are not thread-safe; different sims are.
 */
#ifndef GB300_LBM_H
#define GB300_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_sim lbm_sim;     /* opaque, owned by the library */
typedef struct lbm_batch lbm_batch; /* opaque, owned by the library */

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = 1,         /* invalid argument (null pointer, bad size, bad enum)   */
  LBM_ERR_STATE = 2,       /* call not valid in the simulation's current state       */
  LBM_ERR_OOM = 3,         /* device allocation failed                               */
  LBM_ERR_CUDA = 4,        /* a CUDA runtime call failed (no device, launch error)   */
  LBM_ERR_NONFINITE = 5,   /* the device saw a non-finite density (run diverged)     */
  LBM_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                          */
  LBM_ERR_UNSUPPORTED = 7  /* valid request this build does not implement            */
} lbm_status;

typedef enum { LBM_BGK = 0, LBM_MRT = 1 } lbm_collision;

/* Storage precision of the populations.  All store the deviation from the rest
 * state, h_i = f_i - w_i.  FP64 collides in FP64; FP32 and FP16DEV collide in
 * FP32 (FP16DEV rounds to nearest-even on store). */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16DEV = 2 } lbm_precision;

typedef enum { LBM_OUTFLOW_ZOUHE = 0, LBM_OUTFLOW_NN = 1, LBM_OUTFLOW_CBC = 2 } lbm_outflow_kind;

/* Cell kinds used by lbm_set_geometry. */
enum { LBM_CELL_FLUID = 0, LBM_CELL_SOLID = 1, LBM_CELL_WALL = 2 };

/* Optional device allocator (for instance backed by a framework's caching
 * allocator).  alloc returns NULL on failure (the call then fails with
 * LBM_ERR_OOM and frees what it had taken); free accepts what alloc gave.
 * The library frees a block only after the work that used it has completed
 * on the device, so a pool may hand it out again at once. */
typedef struct {
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* ctx;
} lbm_allocator;

/* Process-wide default allocator (the paper has no counterpart): every device
 * allocation made for a call that names no allocator of its own goes through
 * it -- sims created with lbm_config.alloc NULL (populations, geometry, force
 * ring, scratch) and their batches, the autotuner's scratch, and the scratch of
 * the training and statistics calls.  The struct is copied; NULL restores
 * cudaMalloc / cudaFree.  A sim keeps the allocator it was created with.  The
 * Python binding installs one backed by PyTorch's caching allocator. */
lbm_status lbm_set_default_allocator(const lbm_allocator* alloc);

typedef struct {
  int32_t nx, ny;           /* lattice size; nx >= 3 (>= 5 for NN/CBC outflow) unless x_periodic;
                               ny <= 65535, 9 * ny * pitch < 2^31 (pitch = nx rounded up to 64) */
  double tau;               /* BGK relaxation time (Eq. 2), tau > 1/2; nu = (tau - 1/2) / 3 */
  int32_t collision;        /* lbm_collision */
  double mrt_rates[9];      /* MRT rates in moment order (rho, e, eps, jx, qx, jy, qy, pxx, pxy),
                               each in [0, 2) (else LBM_ERR_ARG); the conserved ones (0, 3, 5)
                               are ignored, the other six relax their moments independently;
                               a zero stress rate (7 or 8) means 1/tau.  All nine zero: e, eps,
                               q rates 1, stress rates 1/tau. */
  int32_t precision;        /* lbm_precision */
  int32_t x_periodic;       /* 1: x wraps too (no inlet, no outflow); 0: open in x */
  double u_in;              /* west inlet velocity (Zou & He, Sec. 2.2 "by symmetry") */
  double v_pert_amp;        /* amplitude of the seeded inlet v perturbation */
  uint64_t seed;            /* v(y,t) = amp (2 xi - 1), xi from SplitMix64(seed ^ (t 2^20 + y)) */
  double rho_out;           /* outflow density for Zou & He (Eq. 7) */
  void* stream;             /* cudaStream_t to run on; NULL: the library creates one */
  const lbm_allocator* alloc; /* NULL: cudaMalloc / cudaFree */
  int64_t force_capacity;   /* device ring of per-step forces (steps); 0: the ring starts at
                               4096 steps and doubles, up to 2^20, before a run of steps would
                               overwrite forces not yet drained by lbm_forces */
  int64_t ramp_steps;       /* > 0: the inlet velocity of step t is u_in min(1, (t+1)/ramp_steps)
                               (a smooth start; the paper does not state how its runs start) */
  int32_t layout;           /* lbm_layout: LBM_LAYOUT_AB (default) or LBM_LAYOUT_AA */
} lbm_config;

/* Population storage.  AB: two buffers, each step pulls from one into the
 * other.  AA (Bailey et al., ICPP 2009): one buffer updated in place, half the
 * population memory for the same 72 B (FP32) of traffic per node and step.
 * Steps from an even step count read every node's nine incoming populations
 * from its neighbours' opposite slots and push the nine outgoing ones into
 * them; steps from an odd count read and write the node's own slots.  Solid
 * nodes need no writes (the swapped slots already hold the reversed
 * populations) and the momentum exchange is summed at the fluid side of each
 * counted link.  Results equal the AB step's (forces up to the summation
 * order).  An AA lattice runs alone (no batches), with the Zou & He outflow,
 * on its own kernels (tiling variants 0-2: the register kernel at three
 * occupancies; 3: a staged kernel, one block per strip, whose producer warp
 * copies each row's source segments into shared memory with cp.async.bulk;
 * the autotuner tries those four; variants 4-6 return LBM_ERR_UNSUPPORTED),
 * and supports neither capture calls nor lbm_copy_columns; one ghost column on
 * each side keeps the populations that leave the lattice, so exports stay
 * exact. */
typedef enum { LBM_LAYOUT_AB = 0, LBM_LAYOUT_AA = 1 } lbm_layout;

/* Fill *cfg with defaults (tau 0.6, BGK, FP32, open x, rho_out 1). */
lbm_status lbm_config_default(lbm_config* cfg);

/* Create a simulation: allocates two population buffers of
 * 9 * ny * pitch elements (pitch = nx rounded up to 64), or with
 * LBM_LAYOUT_AA one buffer with pitch = nx + 2 rounded up to 64, initialised
 * to the rest state (rho = 1, u = 0), all cells fluid, Zou & He outflow. */
lbm_status lbm_create(const lbm_config* cfg, lbm_sim** out);
lbm_status lbm_destroy(lbm_sim* sim);

/* Cell kinds, host uint8[ny][nx]: 0 fluid, 1 solid counted in the force,
 * 2 solid not counted (channel walls).  Solid nodes use full-way bounce-back
 * (Eq. 11).  A counted link joins a kind-1 node s and a fluid node s - c_i
 * (x wraps only if x_periodic; y always wraps). */
lbm_status lbm_set_geometry(lbm_sim* sim, const uint8_t* kind);

/* Set every node to f^eq(rho, ux, uy) (Eq. 3), host double[ny][nx] each;
 * NULL means rho = 1 or u = 0.  Resets the step counter, the force series and
 * the boundary state. */
lbm_status lbm_init_equilibrium(lbm_sim* sim, const double* rho, const double* ux,
                                const double* uy);

/* Outflow by Zou & He with prescribed density (Sec. 2.2, Eqs. 5-10): rho_out,
 * u from Eq. 7, zero tangential velocity. */
lbm_status lbm_set_outflow_zouhe(lbm_sim* sim, double rho_out);

/* A small fully connected network: n_layers layers, layer l maps sizes[l] ->
 * sizes[l+1]; hidden layers apply act (0 tanh, 1 LeakyReLU slope 0.01), the
 * last is linear.  params holds, per layer, W (row-major, sizes[l+1] x
 * sizes[l]) then b.  Inputs are z-scored with in_mean / in_std (NULL: 0 / 1)
 * before the first layer and the output is multiplied by out_scale.
 * All pointers are host memory and are copied. */
#define LBM_MLP_MAX_LAYERS 4
typedef struct {
  int32_t n_layers;
  int32_t sizes[LBM_MLP_MAX_LAYERS + 1];
  int32_t act;
  const float* params;
  int64_t n_params;
  const float* in_mean;
  const float* in_std;
  float out_scale;
} lbm_mlp;

/* Outflow by direct reconstruction (Sec. 3.1, Eq. 15): for every east node,
 * s = net(81 inputs), g_i(L) = f_i(L-1) + s_i for i = 3, 6, 7.  The inputs
 * are the nine post-stream populations of columns L-1, L-2, L-3 at rows
 * y-1, y, y+1 (index k*27 + j*9 + i for column L-1-k, row y-1+j).  The net
 * must map 81 -> ... -> 3 with at most 64 units per hidden layer.  A node
 * falls back to Zou & He (rho_out of the config) when an output is not finite,
 * a rebuilt population is negative, or |rho - rho_out| > fallback_drho; the
 * count is reported by lbm_nn_fallbacks.  Needs nx >= 5. */
lbm_status lbm_set_outflow_nn(lbm_sim* sim, const lbm_mlp* net, double fallback_drho);
lbm_status lbm_nn_fallbacks(lbm_sim* sim, int64_t* count);

/* Characteristic outflow (Sec. 4, Eqs. 17-28).  For every east fluid node
 * (L, y), L = nx - 1, each step: rho, u, v (p = rho/3) of the state at t at
 * (L, y), (L-1, y), (L-2, y), (L, y-1), (L, y+1); d/dx one-sided second order
 * over L, L-1, L-2; d/dy central with y periodic (first order towards the
 * fluid next to a solid row, 0 between two solid rows); wave amplitudes
 * L5 = (u + c_s)(p_x + rho c_s u_x), L3 = u v_x and transverse terms T1, T3,
 * T5 (Eqs. 20-25, with d rho/dx read as dp/dx); the incoming amplitude
 * L1 = kappa1 (p - rho_out/3) - kappa2 T1 + T1 (Eq. 26, T1_exact = 0) with
 * kappa1 = sigma (1 - mach^2) c_s / length (Eq. 27; length 0 = nx); one Euler
 * step of Eqs. 17-19 gives the prescribed (rho, u, v) at t+1; the unknowns
 * 3, 6, 7 follow by Zou & He with that state, then f_0 += rho - (rho0 +
 * 2 rho+)/(1 + u) (Eq. 28), or, with exact_mass = 1, += rho (1 + u) - (rho0 +
 * 2 rho+), which makes the node density exactly rho.  The node then collides.
 * tuner (nullable, host memory, copied): an MLP of 1..3 layers mapping the six
 * derivatives (p_x, u_x, v_x, p_y, u_y, v_y), z-scored by in_mean / in_std, to
 * 1 or 2 outputs s (hidden layers of at most 32 units; out_scale ignored):
 * sigma is then sigma * sigmoid(s_0) per node and, with a second output,
 * kappa2 is kappa2 * sigmoid(s_1).  Needs nx >= 4 and an open x direction. */
lbm_status lbm_set_outflow_cbc(lbm_sim* sim, double sigma, double kappa2, double mach,
                               double length, const lbm_mlp* tuner, int32_t exact_mass);

/* ---- Training data and training of the direct-reconstruction network ----
 * (Sec. 3.1: the network learns, from long-domain runs, the populations 3, 6,
 * 7 that cross a truncation plane; loss Eq. 16.)
 *
 * A data-set row is 84 floats: the 81 inputs of Eq. 15 (post-stream
 * populations of columns x_t-1, x_t-2, x_t-3 at rows y-1, y, y+1, index
 * k*27 + j*9 + i, rows wrapping periodically) followed by the post-stream
 * f_3, f_6, f_7 at (x_t, y).  Rows live in DEVICE memory owned by the caller,
 * row-major float[n][84]. */

/* Capture training rows at column x_t (4 <= x_t <= nx-2): during every step
 * t -> t+1 with (t+1) % every == 0 the library writes ny rows (y = 0..ny-1,
 * in order) after streaming and bounce-back, before collision, into dev_rows
 * (device float[cap_rows][84], caller-owned, must stay valid while capturing)
 * starting at row lbm_capture_count.  Capturing stops once the next ny rows
 * would pass cap_rows.  Resets the count.  dev_rows NULL stops capturing.
 * In a batch each member captures on its own. */
lbm_status lbm_capture_plane(lbm_sim* sim, int32_t x_t, int32_t every, float* dev_rows,
                             int64_t cap_rows);

/* Training rows from one snapshot (Sec. 3.1: the network is trained on a
 * snapshot of a converged flow, each layer of the training region one
 * batch): for every column x in [x_begin, x_end) (4 <= x_begin < x_end <=
 * nx-1) and every row y, the row that lbm_capture_plane at x_t = x would
 * record during the next step (post-stream populations pulled from the current
 * post-collision state, solid nodes reversing what arrives), written to
 * dev_rows[(x - x_begin) * ny + y] (device float[(x_end - x_begin) * ny][84],
 * caller-owned).  Enqueued on the sim's stream; the state is not changed. */
lbm_status lbm_capture_snapshot(lbm_sim* sim, int32_t x_begin, int32_t x_end, float* dev_rows);
/* Rows captured so far (complete once the sim's stream reaches them). */
lbm_status lbm_capture_count(lbm_sim* sim, int64_t* rows);

/* Checkpoint of the simulation state (the paper has no counterpart; a restart
 * facility for long runs): lbm_save writes the current populations (storage
 * precision, the padded layout) and the step counter to a file (host path,
 * created or truncated) after the stream's pending work; lbm_load reads one into
 * a sim created with the same nx, ny and precision (else LBM_ERR_ARG) and sets
 * its step counter, so stepping on gives the same bits as the uninterrupted run.
 * Geometry, outflow settings and networks are not stored: set them as before.
 * The force series restarts empty at the loaded step (drain it before saving). */
lbm_status lbm_save(lbm_sim* sim, const char* path);
lbm_status lbm_load(lbm_sim* sim, const char* path);

/* Normalisation of the network from a data set (device rows, n >= 1): per
 * input the mean and the population standard deviation (a std below 1e-12
 * becomes 1), and out_scale = the population standard deviation of the
 * residual targets f_ref - f_{3,6,7}(x_t - 1) (inputs 12, 15, 16) pooled over
 * the three outputs (same floor).  FP64 sums in a fixed order.  Outputs are
 * host float[81], float[81], float[1].  Synchronous on stream (cudaStream_t,
 * NULL = legacy default stream). */
lbm_status lbm_nn_dataset_stats(const float* dev_rows, int64_t n_rows, void* stream,
                                float* in_mean, float* in_std, float* out_scale);

/* Options of lbm_nn_train / lbm_nn_loss_grad. */
typedef struct {
  int32_t batch_rows;   /* rows per Adam step; batch b = rows [b*batch_rows, (b+1)*batch_rows) */
  double lr;            /* Adam (Kingma & Ba 2015): step size, default 1e-5 */
  double beta1, beta2;  /* default 0.9, 0.999 */
  double eps;           /* default 1e-8 */
  int64_t adam_t0;      /* Adam steps already taken with the given moments (bias correction) */
  int32_t max_cluster;  /* CTAs of the training cluster, 1..16; 0 = the largest that fits */
  void* stream;         /* cudaStream_t; NULL = legacy default stream */
} lbm_train_opts;

/* batch_rows 0, lr 1e-5, beta1 0.9, beta2 0.999, eps 1e-8, adam_t0 0,
 * max_cluster 0, stream NULL. */
lbm_status lbm_train_opts_default(lbm_train_opts* opts);

/* Train net (81 -> ... -> 3, hidden layers of 1..64 units, act tanh or leaky)
 * with Eq. 16: L = mean over the batch and the three outputs of
 * (f_{3,6,7}(x_t-1) + out_scale * o - f_ref)^2, one Adam step per entry of
 * order (host int32[n_steps], batch indices, each in [0, n_rows/batch_rows)).
 * net->in_mean / in_std / out_scale are used as given.  On return params_out
 * (host float[n_params]) holds the trained parameters; adam_m / adam_v (host
 * float[n_params], nullable = zeros in and not returned) are the first and
 * second moments, in and out; loss_log (host double[n_steps], nullable) gets
 * each batch's loss before its step.  FP32 arithmetic, FP64 loss sums.
 * Synchronous.  Runs as one thread-block cluster; results are bitwise
 * reproducible for a given cluster size. */
lbm_status lbm_nn_train(const float* dev_rows, int64_t n_rows, const int32_t* order,
                        int64_t n_steps, const lbm_train_opts* opts, const lbm_mlp* net,
                        float* params_out, float* adam_m, float* adam_v, double* loss_log);

/* Loss of Eq. 16 (host double[n_batches], required) and, if grads is not
 * NULL, its gradient with respect to every parameter (host
 * float[n_batches][n_params], the layout of lbm_mlp.params) for each batch
 * index in order (host int32[n_batches]); no update.  Synchronous. */
lbm_status lbm_nn_loss_grad(const float* dev_rows, int64_t n_rows, const int32_t* order,
                            int64_t n_batches, const lbm_train_opts* opts, const lbm_mlp* net,
                            double* losses, float* grads);

/* ---- Training the CBC tuner through short simulation segments (Sec. 4.2) ----
 * A segment starts from a reference state of the truncated lattice (nx x ny,
 * BGK with tau, y periodic, no solid nodes, east column L = nx - 1 with the
 * characteristic outflow of lbm_set_outflow_cbc and the tuner), runs n_t steps
 * and is compared with the reference state n_t steps later over the last n_t
 * columns (x = L - n_t + 1 .. L, all rows):
 *   loss = mean (rho - rho_ref)^2 + mean over nodes and both components
 *          (U - U_ref)^2,
 * rho and U being the moments of the stored populations.  A batch's loss is
 * the mean of its segments' losses.  Those columns at t0 + n_t depend only on
 * the last W = max(2 n_t, 3) columns at t0 (so the west inlet never enters),
 * and the library runs each segment on that strip alone.  The gradient with
 * respect to the tuner's parameters is the exact reverse-mode derivative of
 * that computation in the chosen precision (adjoint stream-and-collide steps,
 * forward-mode dual numbers for the east node), summed in a fixed order
 * (bitwise reproducible). */
typedef struct {
  int32_t nx, ny;           /* truncated lattice; nx >= W + 1, 3 <= ny <= 65535 */
  int32_t n_t;              /* steps per segment, >= 1 */
  double tau, rho_out;      /* BGK relaxation time (> 1/2); outflow far-field density */
  double sigma, kappa2, mach, length;  /* as lbm_set_outflow_cbc (length 0 = nx) */
  int32_t exact_mass;       /* f_0 correction: 0 Eq. 28, 1 exact mass */
  int32_t precision;        /* LBM_FP64 (default), or LBM_FP32: states, adjoints and the
                               tuner in FP32 on shifted populations h = f - w (loss,
                               parameter sums and Adam stay FP64) */
  const double* bank;       /* device, [n_states][9][ny][bank_width]: populations f (not
                               shifted) of the last bank_width columns of the truncated
                               lattice, e.g. written by lbm_copy_columns; caller-owned */
  int32_t n_states, bank_width;   /* W <= bank_width <= nx */
  const int32_t* init_state;      /* host [n_seg]: bank index of each segment's start */
  const int32_t* final_state;     /* host [n_seg]: bank index of its reference at start + n_t */
  int32_t n_seg;                  /* 1..65535 */
  void* stream;             /* cudaStream_t; NULL = legacy default stream */
} lbm_cbc_segments;

/* Copy the populations f = h + w (FP64, not shifted) of columns
 * [x0, x0 + width) of the sim's current state, every row, into device memory
 * dev_out [9][ny][width] (caller-owned, 9 ny width doubles).  Enqueued on the
 * sim's stream; LBM_ERR_ARG if the columns leave the lattice. */
lbm_status lbm_copy_columns(lbm_sim* sim, int32_t x0, int32_t width, double* dev_out);

/* Normalisation of the tuner's inputs from the bank: per feature (p_x, u_x,
 * v_x, p_y, u_y, v_y at the east column of every bank state, derivatives as in
 * lbm_set_outflow_cbc with y periodic) the mean and the population standard
 * deviation (below 1e-12: 1), FP64 sums in a fixed order, returned as host
 * float[6] each.  Uses bank, n_states, ny, bank_width (>= 3) and stream of segs.
 * Synchronous. */
lbm_status lbm_cbc_feature_stats(const lbm_cbc_segments* segs, float* in_mean, float* in_std);

/* Mean loss over all n_seg segments (host double[1]) and, if grad is not
 * NULL, its gradient with respect to the tuner's parameters (host
 * double[n_params], the layout of lbm_mlp.params), evaluated at params (host
 * double[n_params]).  tuner gives the architecture (6 -> 1..2, 1..3 layers,
 * hidden layers of at most 32 units, act 0 tanh / 1 leaky) and in_mean /
 * in_std (NULL = 0 / 1); tuner->params is ignored.  Allocates its scratch
 * (about n_seg (n_t + 4) 9 ny W doubles), synchronous. */
lbm_status lbm_cbc_segment_grad(const lbm_cbc_segments* segs, const lbm_mlp* tuner,
                                const double* params, double* loss, double* grad);

/* n_steps Adam steps (Kingma & Ba 2015, lr / beta1 / beta2 / eps / adam_t0 /
 * stream of opts; batch_rows and max_cluster are ignored) on the segment loss:
 * step k uses the batch of segments order[k*batch .. (k+1)*batch) (host
 * int32, indices into the segment list).  params (host double[n_params]) is
 * the starting point and receives the result; adam_m / adam_v (host
 * double[n_params], nullable = zeros in and not returned) are the moments, in
 * and out; loss_log (host double[n_steps], nullable) gets each batch's loss
 * before its step.  Synchronous. */
lbm_status lbm_cbc_tuner_train(const lbm_cbc_segments* segs, const lbm_mlp* tuner,
                               const int32_t* order, int32_t batch, int64_t n_steps,
                               const lbm_train_opts* opts, double* params, double* adam_m,
                               double* adam_v, double* loss_log);

/* Enqueue n time steps (n >= 0).  Each step: pull streaming (Eq. 1), momentum
 * exchange (Eqs. 13-14) and bounce-back (Eq. 11) at solid nodes, the west
 * inlet, the east outflow, and collision of all fluid nodes; the force on
 * kind-1 nodes is appended to the device force ring. */
lbm_status lbm_step(lbm_sim* sim, int64_t n);

/* Wait for the stream; report a latched device fault. */
lbm_status lbm_sync(lbm_sim* sim);

/* Number of completed steps. */
lbm_status lbm_time(lbm_sim* sim, int64_t* t);

/* Drain the force series: writes up to cap per-step forces (F_x, F_y, lattice
 * units, F = Delta P / Delta t of Eqs. 13-14) recorded since the previous
 * drain, oldest first, and sets *n_out.  If more steps than the ring holds ran
 * since the previous drain, only the newest ring-capacity entries remain. */
lbm_status lbm_forces(lbm_sim* sim, double* fx, double* fy, int64_t cap, int64_t* n_out);

/* Macroscopic fields rho, ux, uy (Eq. 4), host double[ny][nx] each (any may
 * be NULL).  At solid nodes these are moments of what bounce-back stored. */
lbm_status lbm_fields(lbm_sim* sim, double* rho, double* ux, double* uy);

/* Read / write the populations f_i (not shifted), host double[9][ny][nx].
 * lbm_get_populations returns the post-collision state of the last step. */
lbm_status lbm_get_populations(lbm_sim* sim, double* f);
lbm_status lbm_set_populations(lbm_sim* sim, const double* f);

/* Total mass: sum of every population on every node, accumulated in FP64. */
lbm_status lbm_mass(lbm_sim* sim, double* mass);

/* Device pointer of the current population buffer and its geometry, for
 * zero-copy access: element (i, y, x) is at base[i * plane + y * pitch + x],
 * storing f_i - w_i in the configured precision.  With LBM_LAYOUT_AA after
 * an even number of steps f_i(x, y) is at slot opp(i) of (x, y); after an odd
 * number it is at slot i of (x + c_ix, y + c_iy) (y periodic, x = -1 and
 * x = nx are the ghost columns).  Valid until the next call that steps or
 * destroys the sim. */
lbm_status lbm_device_state(lbm_sim* sim, void** base, int64_t* pitch, int64_t* plane);

/* Tiling of the step kernel: rows per strip (1..4096; a strip is 128 columns)
 * and variant: 0..2 = the register-pipelined kernel on a persistent grid with
 * at least 6, 8 or 10 resident blocks of 128 threads per SM; 3 = the staged
 * kernel (a producer warp copies rows into a shared-memory ring with
 * cp.async.bulk -- with FP16 storage whole input rows of all nine populations,
 * one tensor copy each -- and four consumer warps collide from it; one block
 * per strip);
 * 4 = the staged kernel on a resident-sized grid, each block streaming a
 * fixed share of the strips through its ring; 5 = the staged kernel on a
 * resident-sized grid whose blocks take strips from a global counter (dynamic
 * balance; the counter is reset by the last block, so launches of one sim or
 * batch must not overlap); 6 = variant 3 ordered by per-strip completion
 * flags instead of whole launches: a strip's step waits only for the 3 x 3
 * strips around it to finish the previous step, so the next step's blocks
 * fill the GPU while one step drains (waits give up after 2 s and latch
 * LBM_ERR_TIMEOUT; the east boundary blocks of the NN and characteristic
 * outflows take part with flags of their own; inside a caller's stream
 * capture it runs as variant 3).  Staged variants need rows >= 2.
 * Populations do not depend on the tiling; the FP64 force sum may differ in
 * its last bits (partial sums change order). */
lbm_status lbm_set_tiling(lbm_sim* sim, int32_t rows, int32_t variant);
lbm_status lbm_get_tiling(lbm_sim* sim, int32_t* rows, int32_t* variant);

/* Test hook for the bounded waits of the dataflow order (variant 6; no
 * counterpart in the paper).  With hold != 0 the flags that the sim's next
 * launches start from (after a reset) claim one step fewer than has completed,
 * so no block's wait can be satisfied: each gives up after 2 s, the blocks
 * finish their strips anyway, and the step latches LBM_ERR_TIMEOUT, which
 * lbm_sync reports; the device stays usable.  hold = 0 restores normal resets.
 * LBM_ERR_STATE unless the sim's own tiling is variant 6. */
lbm_status lbm_debug_hold_dataflow(lbm_sim* sim, int32_t hold);

/* Autotuner: time `steps` (1..10000) steps of every candidate tiling (rows 2,
 * 4, 8, 12, 16, 20, 24, 32, 40, 48, 64, 80, 96, 128 x the seven variants) with
 * CUDA events on the sim's stream, back to back as a run executes them, and keep the fastest;
 * *best_ms (nullable) gets its mean step time.  With flush_bytes > 0 a scratch
 * buffer of that size is written before each step, which is then timed alone,
 * so every step starts from a cold L2.  The populations, step
 * counter, force series and fallback count are restored afterwards.  Uses
 * temporary device memory (one population buffer + flush_bytes). */
lbm_status lbm_autotune(lbm_sim* sim, int32_t steps, int64_t flush_bytes, float* best_ms);

/* One FP32 time step of a lattice whose buffers the caller owns, without any
 * device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory themselves or let a library
 * do it -- code recording a CUDA stream capture that must not contain
 * allocations, frameworks whose pool owns all device memory, real-time loops
 * that forbid allocator calls after start-up.
 *
 * It applies the same step as lbm_step with the Zou & He outflow (or periodic
 * x): src -> dst, both device float[9][ny][pitch] holding h_i = f_i - w_i;
 * kind is a device uint8[ny][nx] of cell kinds as for lbm_set_geometry; t is
 * the step index (it keys the seeded inlet perturbation); force is a device
 * double[2] that receives (F_x, F_y) of the step.  From cfg it uses nx, ny,
 * tau, collision, mrt_rates, x_periodic, u_in, v_pert_amp, seed, rho_out,
 * ramp_steps and stream (NULL: the legacy default stream); precision must be LBM_FP32 and
 * alloc and force_capacity are ignored.  The call only enqueues work and
 * reports launch errors; it does not synchronise.
 *
 * Scratch: the per-block force partials live in a 128 KiB static device
 * array that every GPU loading the library holds until exit, so the lattice
 * may have at most 8192 strips of 128 x 8 nodes (8,388,608 nodes); larger
 * lattices are rejected with LBM_ERR_ARG.  Every call made outside a stream
 * capture looks up that array's device address (cudaGetSymbolAddress) with
 * the current device; a call inside a capture reuses the address of the last
 * call on that device, so make the first call on a device before any stream
 * capture (a captured first call returns LBM_ERR_STATE).  MRT rates outside
 * [0, 2) are rejected with LBM_ERR_ARG as in lbm_create.  All calls share the
 * array: calls that overlap on the GPU (for instance on two streams) race on
 * it and must be ordered by the caller. */
lbm_status lbm_step_noalloc(const lbm_config* cfg, const float* src, float* dst,
                            const uint8_t* kind, int64_t pitch, int64_t t, double* force);

/* Batches.  A batch advances several sims -- of any sizes, relaxation times,
 * collision operators, inlet velocities and outflows -- by one kernel launch
 * per time step (the east boundary blocks of NN and characteristic outflows
 * run inside it), the launch table listing every member's strips; runs of
 * steps are cut into chunks of 32 steps and one of the remaining 4-31 (fewer
 * launch directly) that replay from CUDA graphs (a graph is instantiated the
 * first time its length and starting buffer occur, then reused).  Members must share one precision and one stream
 * (lbm_config.stream) and be at the same step (for instance all freshly
 * initialised); the batch keeps them in lockstep.  Members remain ordinary
 * sims for every other call (lbm_forces, lbm_fields, ...); stepping a member
 * alone breaks the lockstep, after which lbm_batch_step reports
 * LBM_ERR_STATE.  Destroy batches before their members.  The batch allocates
 * its own launch table and force partials.  sims is a host array of n >= 1
 * distinct sims (copied). */
lbm_status lbm_batch_create(lbm_sim* const* sims, int32_t n, lbm_batch** out);
lbm_status lbm_batch_destroy(lbm_batch* batch);
lbm_status lbm_batch_step(lbm_batch* batch, int64_t n);
/* Wait for the stream; report the first latched device fault of any member. */
lbm_status lbm_batch_sync(lbm_batch* batch);
/* Tiling and autotuner of the batch launch, as lbm_set_tiling / lbm_autotune
 * (in a batch every variant launches one block per strip). */
lbm_status lbm_batch_set_tiling(lbm_batch* batch, int32_t rows, int32_t variant);
lbm_status lbm_batch_get_tiling(lbm_batch* batch, int32_t* rows, int32_t* variant);
lbm_status lbm_batch_autotune(lbm_batch* batch, int32_t steps, int64_t flush_bytes,
                              float* best_ms);

/* Strouhal number of a lift series (Sec. 2.3): St = f D / U with f the peak of
 * |DFT| of the last 2^m samples (largest power of two <= n, n >= 8), mean
 * removed, Hann window, refined by a parabola through the peak bin and its
 * neighbours.  Host-only; needs no device. */
lbm_status lbm_strouhal(const double* cl, int64_t n, double length, double u, double* st);

/* Message of the last failed call on this thread ("" if none). */
const char* lbm_last_error(void);

/* Library version string. */
const char* lbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GB300_LBM_H */
