/*
 * bsparareal.h -- C ABI of the B300 (sm_103a) Parareal/PINN library for the
 * Black-Scholes European call.
 *
 * Method: Ibrahim, Goetschel, Ruprecht, "Parareal with a physics-informed
 * neural network as coarse propagator" (arXiv:2303.03848).
 *   - PDE: Eq. 1 (Section 3), solved in time-to-maturity tau = T - t, with the
 *     payoff (Eq. 2) as initial value and Dirichlet values V(tau, 0) = 0 (Eq. 3),
 *     V(tau, Smax) = Smax - K exp(-r tau) (far-field reading of Eq. 4).
 *   - Space: second-order centred differences on S_j = j dS, j = 0..Nx-1,
 *     dS = Smax / (Nx - 1) (Eqs. 9-10, Section 3.2).
 *   - Fine propagator F: Crank-Nicolson; numerical coarse G: implicit Euler
 *     (Section 3.2).  PINN coarse: a tanh MLP in (S, tau) (Section 3.3).
 *   - Parareal: Eq. 7 (Section 3.1).
 *
 * General conventions
 *   - Every function returns a bs_status (int).  BS_EINVAL means the
 *     arguments were rejected and nothing was launched.  No function aborts.
 *   - Device buffers are owned by the caller, must be 16-byte aligned, dense
 *     and resident on the current CUDA device.  Host buffers are marked "host".
 *   - stream is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on that stream unless stated otherwise.
 *   - Handles (bs_problem, pinn_model) are created and destroyed by the
 *     library.  A handle must not be used from two streams at once.
 *   - Layout of state arrays: instance i owns (P_i + 1) * Nx_i doubles for
 *     slice-boundary states (parareal_solve, serial_fine) or P_i * Nx_i doubles
 *     for slice inputs/outputs (fine_propagate, coarse_propagate), instances
 *     packed back to back in the order given to bs_problem_init; slice n of
 *     instance i is the Nx_i doubles at offset (off_i + n * Nx_i).
 */
#ifndef BSPARAREAL_H
#define BSPARAREAL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
  BS_OK = 0,
  BS_EINVAL = 1,          /* invalid argument; nothing launched */
  BS_ECUDA = 2,           /* a CUDA call failed (launch or copy) */
  BS_ENOMEM = 3,          /* device or host allocation failed */
  BS_NOT_CONVERGED = 4,   /* max_iter reached before tol (parareal_solve) */
  BS_DIVERGED = 5,        /* a non-finite value reached the convergence norm */
  BS_TIMEOUT = 6,         /* a bounded device wait gave up */
  BS_EUNSUPPORTED = 7     /* size or mode outside what this build supports */
} bs_status;

/*
 * Coarse propagator kinds for parareal_solve (Sections 3.1 and 3.3).  g_n
 * below is the network table u_theta(S_j, tau_n) with exact Dirichlet nodes.
 * BS_COARSE_PINN_IE reads the network of Section 3.3 / Fig. 2 as a propagator
 * that is given V at t_start: the network's own value at tau_{n+1} plus the
 * implicit Euler response to the deviation of U_n from the network's value at
 * tau_n.  Implicit Euler is affine, so this is IE(U_n) + (g_{n+1} - IE(g_n))
 * at the interior nodes (IE's exact values at the Dirichlet nodes); the
 * corrections g_{n+1} - IE(g_n) are formed once per solve for all slices at
 * once, so each step of the serial sweep costs one IE step and one addition.
 * G(g_n) = g_{n+1}: the network's solution is a trajectory of this G.
 */
typedef enum {
  BS_COARSE_IE = 0,         /* implicit Euler, coarse_steps steps per slice (Section 3.2) */
  BS_COARSE_PINN = 1,       /* G(U_n) = g_{n+1}, independent of U_n */
  BS_COARSE_PINN_INCR = 2,  /* G(U_n) = U_n + g_{n+1} - g_n */
  BS_COARSE_PINN_IE = 3     /* G(U_n) = g_{n+1} + IE response to (U_n - g_n) = IE(U_n) + g_{n+1} - IE(g_n) */
} bs_coarse_kind;

/* Arithmetic of the network evaluation.  Fine/coarse solves are always FP64. */
typedef enum { BS_FP64 = 0, BS_FP32 = 1, BS_TF32 = 2, BS_BF16 = 3 } bs_precision;

/* One pricing instance.  Nx counts grid points including both Dirichlet nodes. */
typedef struct {
  double K, sigma, r, T, Smax;
  int32_t Nx, P, fine_steps, coarse_steps;
} bs_params;

/* Per-instance result of parareal_solve (host). */
typedef struct {
  int32_t iterations;  /* Parareal iterations done (k) */
  int32_t status;      /* bs_status of this instance */
  double final_norm;   /* last increment norm e_k */
} bs_instance_stats;

typedef struct bs_problem bs_problem;
typedef struct pinn_model pinn_model;

/* Text for a status code (static storage). */
const char* bs_status_string(int status);

/* Library version string. */
const char* bs_version(void);

/*
 * bs_wait_probe -- diagnostic of the device-side failure detection: one CTA
 * runs a bounded mbarrier wait the way the tensor-core kernels do (try_wait
 * with an SM clock limit of limit_cycles, 1 .. 2^34) on a barrier that one
 * thread completes (arrive != 0) or that nothing completes (arrive == 0).
 * *status (host) receives BS_OK or BS_TIMEOUT; the context stays usable after
 * a timeout.  Synchronous.  Errors: BS_EINVAL, BS_ECUDA.
 */
int bs_wait_probe(int32_t arrive, int64_t limit_cycles, int32_t* status);

/*
 * bs_problem_init -- set up n_instances pricing problems on the current device.
 *   p: host array of n_instances parameter sets.  Requirements per instance:
 *      K > 0, sigma > 0, r >= 0, T > 0, Smax > K, 5 <= Nx <= 65537, P >= 1,
 *      fine_steps >= 1, coarse_steps >= 1, all finite.
 *   Builds the Eq. 10 coefficients and factorises the Crank-Nicolson matrix
 *   (I - dtau_f/2 L) and the implicit Euler matrix (I - dtau_g L) on the
 *   device (Section 3.2), once; later calls reuse them.
 *   Each grid is laid out over one CTA (one SM) or, when the problem has few
 *   slices or more than 4096 rows, over a cluster of up to 16 CTAs that
 *   exchange interface values through distributed shared memory; the
 *   environment variable BSP_CLUSTER (1, 2, 4, 8, 16) overrides the cluster
 *   size, and BSP_PARTITION="M,NW,C[,S2]" forces one compiled partition (M rows
 *   per thread, NW warps per CTA, C CTAs; S2 = 2 runs two slices of an instance
 *   per CTA in the fine propagation, sharing its tables) on every instance
 *   (BS_EUNSUPPORTED if it is not compiled or holds fewer than Nx - 1 rows);
 *   BSP_S2=2 selects slice pairs wherever the chosen partition supports them.
 *   Synchronous.  *out receives the handle.  Errors: BS_EINVAL (argument),
 *   BS_EUNSUPPORTED (Nx above the largest grid this build keeps on chip),
 *   BS_ENOMEM, BS_ECUDA.
 */
int bs_problem_init(const bs_params* p, int32_t n_instances, bs_problem** out);

/* One timed candidate of bs_problem_init_tuned. */
typedef struct {
  int32_t Nx;            /* grid size the candidate was timed for */
  int32_t M, NW, C;      /* rows per thread, warps per CTA, CTAs per grid */
  int32_t S2;            /* slices per CTA in the fine propagation (1, or 2: slices in pairs) */
  float ms;              /* device time of one fine propagation of the tuning subset */
  int32_t chosen;        /* 1 for the partition kept for this grid size */
} bs_tuning;

/*
 * bs_problem_init_tuned -- bs_problem_init with the partition of every grid
 * size picked by measurement instead of the built-in rule: for each distinct
 * Nx, every compiled partition (M rows per thread x NW warps x C CTAs, and for
 * partitions with 16 or more rows per thread also two slices per CTA) that
 * holds the grid with at most half of its rows padding is set up for a subset
 * of the problem's own instances of that size (enough for >= 4096 slices, fine
 * steps capped at 128) and timed on one fine propagation (CUDA events, best of
 * two after a warm-up); the fastest is kept.  Few slices favour clusters and
 * several warps per grid (latency), many slices one warp per grid with more
 * rows per thread (throughput).  report (host, nullable when report_cap = 0)
 * receives up to report_cap timed candidates and *n_report (nullable) their
 * number.  Synchronous; the tuning runs on the default stream.  Errors as
 * bs_problem_init; BS_TIMEOUT if a timed candidate's exchange wait gave up.
 */
int bs_problem_init_tuned(const bs_params* p, int32_t n_instances, bs_problem** out, bs_tuning* report,
                          int32_t report_cap, int32_t* n_report);

/*
 * bs_problem_init_partitioned -- bs_problem_init with the partition of every
 * grid size given: for each instance the entry of parts (host, n_parts) with
 * the instance's Nx and chosen != 0 (the fields ms are ignored), e.g. the
 * report of an earlier bs_problem_init_tuned kept in a cache.  Synchronous.
 * Errors: BS_EINVAL (argument, or a grid size without a chosen entry),
 * BS_EUNSUPPORTED (a partition not compiled or too small for its grid),
 * BS_ENOMEM, BS_ECUDA.
 */
int bs_problem_init_partitioned(const bs_params* p, int32_t n_instances, const bs_tuning* parts, int32_t n_parts,
                                bs_problem** out);

/* Release the handle and its device memory.  NULL is accepted. */
void bs_problem_destroy(bs_problem* prob);

/* Instance count and the lengths (doubles) of state ((P+1)-slice) and slice (P-slice) arrays. */
int bs_problem_info(const bs_problem* prob, int32_t* n_instances, int64_t* total_state_doubles,
                    int64_t* total_slice_doubles);

/* Partition of instance i's grid: rows per thread M, warps per CTA NW, CTAs per grid C (cluster size). */
int bs_problem_partition(const bs_problem* prob, int32_t i, int32_t* M, int32_t* NW, int32_t* C);

/* Slices per CTA of instance i's fine propagation: 1, or 2 when two slices of the
 * instance share each CTA and its coefficient tables (partitions with 16 or more
 * rows per thread; the built-in rule takes them for clusters, and for one-CTA
 * grids with 32 rows per thread, when the slices keep every CTA busy twice over). */
int bs_problem_slices_per_cta(const bs_problem* prob, int32_t i, int32_t* s2);

/*
 * bs_problem_device_status -- synchronises the device and reports the
 * problem's device status word: BS_OK, or BS_TIMEOUT if a bounded wait of the
 * per-step exchange between the CTAs of a cluster gave up (the results of that
 * call are then invalid).  The word is sticky until the handle is destroyed.
 * parareal_solve and parareal_solve_static return BS_TIMEOUT themselves when
 * they read statistics back.
 */
int bs_problem_device_status(const bs_problem* prob, int* status);

/*
 * fine_propagate -- the fine propagator F of Eq. 6 on every slice at once:
 *   U_out[n] = F_n(U_in[n]): fine_steps Crank-Nicolson steps of
 *   dtau_f = T / (P * fine_steps) from tau_n = n T / P to tau_{n+1}.
 *   U_in, U_out: device, sum_i P_i * Nx_i doubles (slice layout above).
 *   Dirichlet nodes of U_in are ignored (V_0 = 0; the Smax node is taken as
 *   the exact value at tau_n); U_out carries exact Dirichlet values.
 *   active: device, nullable; one byte per (instance, slice) in the same order;
 *   slices with 0 are left untouched in U_out.  U_in and U_out must not overlap.
 */
int fine_propagate(bs_problem* prob, const double* U_in, double* U_out, const uint8_t* active, void* stream);

/*
 * coarse_propagate -- the implicit Euler coarse propagator G on every slice:
 * coarse_steps steps of dtau_g = T / (P * coarse_steps).  Same layout and
 * rules as fine_propagate.
 */
int coarse_propagate(bs_problem* prob, const double* U_in, double* U_out, const uint8_t* active, void* stream);

/*
 * serial_fine -- classical time stepping (Eq. 6 for n = 0..P-1) from the payoff:
 *   U_out[0] = payoff, U_out[n+1] = F_n(U_out[n]).  U_out: device, state layout.
 *   Each slice restarts from the stored vector, so slice n equals
 *   fine_propagate applied to U_out[n-1] bit for bit.
 */
int serial_fine(bs_problem* prob, double* U_out, void* stream);

/*
 * pinn_create -- a fully connected tanh network (Section 3.3) with
 * n_layers linear layers: widths[0] = d_in (2: inputs (S, tau);
 * 5: (S, tau, sigma, r, K)), widths[1..n_layers-1] hidden (<= 256),
 * widths[n_layers] = 1.  Hidden layers use tanh; the output layer is linear.
 * Parameters are laid out per layer as W [w_out][w_in] row-major then b [w_out].
 * Initialisation: Xavier-uniform weights, zero biases, drawn from SplitMix64
 * in counter form (parameter index q uses output q+1 of the sequence started
 * at `seed`; W = (2u - 1) sqrt(6 / (fan_in + fan_out)), u the top 53 bits).
 * in_lo/in_hi (host, d_in each): the input box; inputs are mapped affinely to
 * [-1, 1] inside the model.  Synchronous.
 */
int pinn_create(const int32_t* widths, int32_t n_layers, const double* in_lo, const double* in_hi, uint64_t seed,
                pinn_model** out);
void pinn_destroy(pinn_model* m);
/* Number of parameters (doubles in the flat layout). */
int pinn_num_params(const pinn_model* m, int64_t* n);
/* Copy FP64 parameters in (host), refresh the reduced-precision copies, reset Adam state.  Synchronous. */
int pinn_set_weights(pinn_model* m, const double* flat_host);
/* Copy the FP64 master parameters out (host).  Synchronous. */
int pinn_get_weights(const pinn_model* m, double* flat_host);
/*
 * pinn_get_state / pinn_set_state -- the whole training state, for checkpoint
 * and resume: FP64 master parameters, Adam's first and second moments (host,
 * n_params doubles each) and the Adam step count.  pinn_set_state refreshes
 * the reduced-precision copies; a train step after it continues exactly as
 * after the pinn_get_state it came from.  Synchronous.  Errors: BS_EINVAL
 * (null pointer, non-finite value, negative second moment or step), BS_ECUDA.
 */
int pinn_get_state(const pinn_model* m, double* theta, double* mom1, double* mom2, int64_t* step);
int pinn_set_state(pinn_model* m, const double* theta, const double* mom1, const double* mom2, int64_t step);

/*
 * pinn_device_status -- synchronises the device and reports the network's
 * device status word: BS_OK; BS_TIMEOUT if a bounded wait inside a
 * tensor-core kernel gave up (its results are then invalid); BS_EINVAL if a
 * loss call met a point of a kind outside 0..3, or of kind 4 in a call without
 * values y (such points were left out of that call's loss terms, counts and
 * gradient).  The word is sticky until the handle is destroyed.
 */
int pinn_device_status(const pinn_model* m, int* status);

/*
 * pinn_eval -- u = u_theta(X) at N points (Section 3.3).
 *   X: device [N][d_in] doubles.  u: device [N] doubles.
 *   derivs: device, nullable, [N][3] = (u_S, u_SS, u_tau) by forward-mode
 *   differentiation through every layer (the paper uses automatic
 *   differentiation).  prec selects the arithmetic of the layers: FP64, FP32,
 *   TF32 or BF16 (reduced precisions accumulate in FP32); outputs are FP64.
 *   BF16 runs the hidden layers on the tensor cores (tcgen05 kind::f16, FP32
 *   accumulation in tensor memory) when every hidden layer is w x w with w a
 *   multiple of 32 up to 256; TF32 likewise (kind::tf32, operands rounded to
 *   TF32 with round-to-nearest) for w up to 128; other shapes round the
 *   operands on CUDA cores.
 *   derivs requires FP64 or FP32.
 */
int pinn_eval(const pinn_model* m, int prec, const double* X, int64_t N, double* u, double* derivs, void* stream);

/*
 * pinn_loss_grad -- loss terms and gradient at the current weights, no update.
 * Loss Eq. 11 = MSE_f (Eq. 12, residual u_tau - 1/2 sigma^2 S^2 u_SS - r S u_S + r u)
 *             + MSE_b (Eq. 13) + MSE_exp (Eq. 14), each the mean over its points.
 *   X: device [N][d_in] doubles; kind: device [N] int8: 0 interior,
 *   1 boundary S = 0 (target 0), 2 boundary S = Smax (target Smax - K e^{-r tau}),
 *   3 expiry tau = 0 (target max(S - K, 0)); kind 4 (data point) belongs to
 *   pinn_loss_grad_data.  The kinds live on the device, so this call does not
 *   read them on the host: a point of any other kind (here also 4) is left out
 *   and BS_EINVAL recorded in the network's status word (pinn_device_status).
 *   X and kind hold N entries each (the library cannot check device lengths).
 *   prob_params (host): K, sigma, r,
 *   Smax of the loss (a 5-input network takes sigma, r, K per point from X;
 *   then Smax of kind-2 points is smax_over_K * K when smax_over_K > 0).
 *   prec: BS_FP64, BS_FP32, BS_TF32 or BS_BF16 (TF32 / BF16: operands of
 *   every layer rounded to the type, FP32 accumulation).
 *   loss3 (device, 3 doubles: MSE_f, MSE_b, MSE_exp) and grad (device,
 *   n_params doubles) are written asynchronously.
 *   BF16 and TF32 with hidden layers w x w, w in {32, 64, 96, 128}, at least
 *   two of them, and d_in 2 or 5 run on the tensor cores (other shapes round
 *   the operands the same way on CUDA cores).  BF16 processes the batch in
 *   chunks of 2^19 points (environment variable BSP_TRAIN_CHUNK overrides, in
 *   points), so its workspace does not grow past one chunk's whatever N; the
 *   other precisions keep 8 N (sum of the layer widths) values.  The
 *   workspace is allocated on first use and grown when a larger batch needs
 *   more.
 */
int pinn_loss_grad(const pinn_model* m, const double* X, const int8_t* kind, int64_t N,
                   const bs_params* prob_params, double smax_over_K, int prec, double* loss3, double* grad,
                   void* stream);

/*
 * pinn_train_step -- pinn_loss_grad followed by one full-batch Adam step
 * (Section 3.3; beta1 0.9, beta2 0.999, eps 1e-8, step size lr) on the FP64
 * master parameters.  loss3: host, nullable; if given the call synchronises the
 * stream, stores the loss terms evaluated BEFORE the update and returns the
 * network's status word when it is not BS_OK (BS_EINVAL: a point of an
 * invalid kind was left out).  grad_out: device, nullable, n_params doubles:
 * receives the gradient used.
 */
int pinn_train_step(pinn_model* m, const double* X, const int8_t* kind, int64_t N, const bs_params* prob_params,
                    double smax_over_K, int prec, double lr, double* loss3, double* grad_out, void* stream);

/*
 * pinn_loss_grad_data, pinn_train_step_data -- pinn_loss_grad and
 * pinn_train_step with data points as well (Section 4: a network trained on
 * fine-propagator output alone, without the PDE terms, compared with the PINN).
 * kind 4 marks a data point; its squared misfit (u - y[i])^2 joins the mean of
 * the first loss term, so loss3[0] is the mean over kind-0 residuals and kind-4
 * misfits together (a batch of kind 4 only trains on data alone).
 *   y: device [N] doubles, 8-byte aligned, non-null (read at kind-4 points
 *   only; N entries).  Every other argument, the precisions and the
 *   tensor-core path are those of pinn_loss_grad / pinn_train_step; kinds
 *   outside 0..4 are left out and recorded as there.  BS_EINVAL for a null or
 *   misaligned y.
 */
int pinn_loss_grad_data(const pinn_model* m, const double* X, const int8_t* kind, const double* y, int64_t N,
                        const bs_params* prob_params, double smax_over_K, int prec, double* loss3, double* grad,
                        void* stream);
int pinn_train_step_data(pinn_model* m, const double* X, const int8_t* kind, const double* y, int64_t N,
                         const bs_params* prob_params, double smax_over_K, int prec, double lr, double* loss3,
                         double* grad_out, void* stream);

/*
 * parareal_solve -- Parareal (Eq. 7) on every instance:
 *   U^{k+1}_{n+1} = F(U^k_n) + (G(U^{k+1}_n) - G(U^k_n)),
 * with G chosen by coarse_kind (model required for the network kinds; the
 * network is evaluated once per call in arithmetic prec on (S_j, tau_n) and
 * its Dirichlet nodes replaced by the exact values).  Iteration k runs F on
 * slices n >= k of the instances still iterating only; once none is, the
 * remaining iterations' launches return at once.  Scheduling counters in the
 * problem's device memory are cleared at the start of every call, so calls on
 * one problem must not overlap on the GPU.  Stops per instance when the increment norm
 *   e_k = max_n ||U^{k+1}_n - U^k_n||_2 / ||U^{k+1}_n||_2 <= tol,
 * or k = P (then Parareal equals serial fine), or k = max_iter.
 *   U_out: device, state layout, the final iterate.
 *   norms: host, nullable, n_instances * max_iter doubles (e_k per iteration;
 *   NaN where not run).  stats: host, nullable, n_instances entries.
 * Synchronises the stream before returning when norms or stats is given.
 * Returns BS_OK when every instance converged, else the worst instance status.
 */
int parareal_solve(bs_problem* prob, int coarse_kind, const pinn_model* model, int prec, double tol,
                   int32_t max_iter, double* U_out, double* norms, bs_instance_stats* stats, void* stream);

/*
 * parareal_solve_static -- parareal_solve without any device allocation.
 * The paper has no counterpart: this is a service for callers that must not
 * allocate device memory once their set-up is done, such as code enqueuing
 * work while a stream is being captured, loops where cudaMalloc/cudaFree would
 * synchronise the device and stall other streams, or processes whose device
 * memory is already reserved by another allocator.  (parareal_solve allocates
 * its workspace on the problem handle on its first call.)
 *   Arguments, results and status codes are those of parareal_solve.  The
 *   workspace lives in one fixed 16 MiB device array inside the library (held
 *   on every GPU that loads the library until the process exits): about 5
 *   doubles per value of the state layout, plus d_in more with a network
 *   coarse propagator (for Nx = 1024, P = 32 and a 2-input network, 1.9 MB).
 *   A solve that needs more, or has more than 256 instances, returns
 *   BS_EUNSUPPORTED and launches nothing.
 *   The first call on each device looks up the array's device address; make
 *   that first call before any stream capture.  All calls share the array and
 *   it keeps the last call's contents; each call clears what must start at
 *   zero.  Calls whose GPU work overlaps (different streams or host threads)
 *   race on the array and must be serialised by the caller.
 */
int parareal_solve_static(bs_problem* prob, int coarse_kind, const pinn_model* model, int prec, double tol,
                          int32_t max_iter, double* U_out, double* norms, bs_instance_stats* stats, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BSPARAREAL_H */
