/*
 * fibers.h -- C ABI of the GB300 (sm_103a) fiber monodomain library.
 *
 * The library advances many independent 1D muscle fibers through the
 * operator-split monodomain model of Maier 2021 ("Scalable Biophysical
 * Simulations of the Neuromuscular System"):
 *
 *   dV/dt = (sigma_eff d2V/dx2 - Am I_ion(V, y)) / (Am Cm)   (eq:monodomain)
 *
 * with homogeneous Neumann ends (eq:monodomain_bc1), the Hodgkin-Huxley
 * subcellular model (sec:subcelullar_model, eq:subcellular), lumped-mass
 * linear finite elements (sec:mass_lumping), Crank-Nicolson diffusion
 * (eq:lumping_crank_nicolson_2) solved per fiber as a tridiagonal system
 * (sec:improved_parallel_solver_for_fiber_based), Heun reaction steps
 * (eq:heun) and Strang splitting (eq:monodomain_strang): per split step
 * dt_split one diffusion half (dt_split/2), the reaction over dt_split in
 * Heun substeps of dt_0d, and a second diffusion half.  Fibers are driven by
 * motor-unit (MU) firing trains at their neuromuscular junction
 * (sec:stimulation_times_callbacks).
 *
 * Units: cm, ms, mV, uA/cm^2, uF/cm^2, mS/cm^2, mS/cm.
 *
 * Conventions for every call:
 *   - Every function returns a fib_status; nothing throws across the ABI.
 *     A failing call leaves a message readable with fibers_last_error().
 *   - The library copies every input array; the caller keeps ownership of
 *     its buffers.  A context owns all device memory it allocates and frees
 *     it in fibers_destroy().
 *   - Work is enqueued on the stream given to fibers_create (NULL: the
 *     legacy default stream).  step() is asynchronous; errors raised by the
 *     device (non-finite state) are reported by the next synchronising call
 *     (read_vm, fibers_read_state, fibers_synchronize, fibers_stats).
 *   - Node arrays are in "ragged order": the nodes of fiber 0, then fiber 1,
 *     and so on, sum(n_nodes) entries in total.
 *   - A context is used by one host thread at a time.
 */
#ifndef FIBERS_H_
#define FIBERS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fib_ctx fib_ctx;

typedef enum {
  FIB_OK = 0,
  FIB_EINVAL = 1,      /* bad argument (message says which) */
  FIB_ENOMEM = 2,      /* device or host allocation failed */
  FIB_ECUDA = 3,       /* a CUDA runtime call failed (message has the CUDA error) */
  FIB_ENONFINITE = 4,  /* the state became NaN/Inf; it stays readable */
  FIB_ETIMEOUT = 5,    /* a bounded wait gave up (on the host, or between a kernel's warps) */
  FIB_ESTATE = 6,      /* call not valid in the current state */
  FIB_ENOTSUP = 7,     /* valid request that the library does not support */
  FIB_EIO = 8          /* a file could not be opened, read or written */
} fib_status;

/* Solve modes. */
enum {
  FIB_MODE_FP32 = 0,         /* FP32 state and arithmetic */
  FIB_MODE_FP64_THOMAS = 1,  /* FP32 state and reaction; tridiagonal solve in FP64 */
  FIB_MODE_SURROGATE = 2     /* reaction step by a learned MLP with HH fallback */
};

/* Flags (fib_params.flags). */
enum {
  /* Adaptive computation (sec:adaptive_computation_for_fiber_based): a fiber
   * whose every node passed the thesis's equilibrium test over the last split
   * step of a kernel launch (each of V, m, h, n changed by at most 1e-5
   * relative) and whose motor unit has no stimulus pulse overlapping the next
   * launch is not computed during that launch (steps_per_launch split steps).
   * All fibers start active.  Not available with FIB_MODE_SURROGATE. */
  FIB_FLAG_ADAPTIVE = 1,
  /* The thesis's approximated exponential (eq:apx-e-function): every
   * exponential of the HH rate formulas is evaluated as exp*(x) =
   * (1 + x/1024)^1024, on the FP32 pipe instead of the special-function
   * unit.  It changes the model (relative error of exp* below 0.07 for
   * |x| < 12), so the rest state and the derived leak reversal follow the
   * approximated rates.  FIB_MODE_FP32 only. */
  FIB_FLAG_EXP_APPROX = 2
};

/* Operator-splitting orderings (fib_params.splitting).  The splitting
 * equations name the diffusion operator L1, so they read diffusion first;
 * the splitting figures order the substeps reaction first.  Both are offered.
 * Reaction phases are whole Heun substeps of dt_0d, diffusion phases whole
 * steps of dt_1d. */
enum {
  FIB_SPLIT_STRANG_1D0D1D = 0,  /* diffusion dt/2, reaction dt, diffusion dt/2 (eq:monodomain_strang) */
  FIB_SPLIT_GODUNOV_1D0D = 1,   /* diffusion dt, reaction dt (eq:monodomain_godunov) */
  FIB_SPLIT_STRANG_0D1D0D = 2,  /* reaction dt/2, diffusion dt, reaction dt/2 (fig:strang_splitting);
                                   dt_split / dt_0d must be even */
  FIB_SPLIT_GODUNOV_0D1D = 3    /* reaction dt, diffusion dt (fig:godunov_splitting) */
};

/* Diffusion time-stepping method (fib_params.diffusion). */
enum {
  FIB_DIFFUSION_CRANK_NICOLSON = 0,  /* (I - dt/2 M^-1 K) u+ = (I + dt/2 M^-1 K) u (eq:lumping_crank_nicolson_2) */
  FIB_DIFFUSION_IMPLICIT_EULER = 1   /* (I - dt M^-1 K) u+ = u (eq:lumping_implicit_euler_2) */
};

/* Model and discretisation parameters (sec:subcelullar_model, eq:monodomain,
 * eq:monodomain_strang).  ENa, EK and EL are absolute reversal potentials;
 * EL = NaN asks the library to derive it so that (Vrest, m_inf, h_inf, n_inf)
 * is an exact rest state.  The HH rates are those of Hodgkin & Huxley 1952 in
 * the depolarisation u = V - Vrest.  dt_split / dt_0d must be a whole number,
 * and so must the diffusion phase's length over dt_1d: (dt_split/2) / dt_1d
 * for FIB_SPLIT_STRANG_1D0D1D, dt_split / dt_1d for the other orderings.
 * FIB_MODE_SURROGATE takes only the default ordering and Crank-Nicolson.
 * A firing at time t_f switches the stimulus
 * on for Heun substeps k with k_f <= k < k_f + P, k_f = round(t_f / dt_0d)
 * (half to even), P = round(stim_duration / dt_0d), at junction nodes
 * j - stim_half_width .. j + stim_half_width (clipped to the fiber).  */
typedef struct {
  double Cm, gNa, gK, gL, ENa, EK, EL, Vrest;
  double sigma_eff, Am, h;
  double dt_split, dt_0d, dt_1d;
  double stim_amplitude, stim_duration;
  int32_t stim_half_width;
  int32_t mode;     /* FIB_MODE_* */
  int32_t flags;     /* FIB_FLAG_* bits (0: none) */
  int32_t splitting; /* FIB_SPLIT_* (0: Strang, diffusion first) */
  int32_t diffusion; /* FIB_DIFFUSION_* (0: Crank-Nicolson) */
  int32_t reserved;  /* must be 0 */
} fib_params;

/* Launch shape.  Zero fields mean "choose automatically". */
typedef struct {
  int32_t nodes_per_thread;  /* K: 4, 8, 12 or 16 nodes held in registers per thread */
  int32_t warps_per_cta;     /* CTA size in warps (1..32); fibers are packed by whole warps */
  int32_t steps_per_launch;  /* split steps each kernel launch keeps on chip */
  int32_t graph_steps;       /* split steps per captured CUDA graph (0 = no graphs) */
  int32_t reaction_pairs;    /* 1: one node per FP32 instruction; 2: node pairs with packed
                                FP32x2 instructions (same results bit for bit); 0: automatic */
  int32_t ctas_per_sm;       /* register budget of the step kernel, as CTAs of 256 threads per
                                SM: 2 (up to 128 registers per thread), 3 (up to 80) or 4 (up to
                                64, more warps per SM, a few spills at K = 8); 0: automatic */
  int32_t warp_roles;        /* 1: every warp of a fiber runs both the reaction and the diffusion
                                solve (the fused kernel); 2: split roles, with 12 reaction warps
                                (4 nodes per lane) and 4 diffusion warps (12 nodes per lane)
                                per CTA of two fibers held in shared memory; 3: split roles in
                                one 1024-thread CTA per SM of eight fibers, 24 reaction warps (8
                                nodes per lane) and two groups of 4 diffusion warps.  2 and 3
                                apply to fibers of at most 1536 nodes in FIB_MODE_FP32 with no
                                flags, Strang 1D-0D-1D and Crank-Nicolson (nodes_per_thread,
                                warps_per_cta, reaction_pairs and ctas_per_sm then do not
                                apply); 0: automatic */
} fib_tuning;

/* Creates a context for n_fibers fibers and copies the inputs to the device.
 *   p             model parameters (copied).
 *   n_fibers      >= 0.
 *   n_nodes       [n_fibers] nodes per fiber, >= 1 (mesh width p->h).
 *   mu_of_fiber   [n_fibers] motor unit of each fiber, or -1 (never stimulated).
 *   junction_node [n_fibers] neuromuscular-junction node, 0 <= j < n_nodes.
 *   vm0           [sum(n_nodes)] initial V in mV, or NULL for V = Vrest.
 *                 Gates start at their steady state at Vrest.
 *   tuning        launch shape, or NULL for automatic.
 *   cuda_stream   cudaStream_t to run on, or NULL.
 *   out           receives the context (NULL on failure).
 * Errors: FIB_EINVAL (bad parameter, fiber too long for the tuning),
 * FIB_ENOMEM, FIB_ECUDA.  Thesis: the inputs FastMonodomainSolver sends to
 * the GPU once (section "Code Generation for GPUs": initial state, junctions, fiber
 * to MU map) and eq:discretized_fibers (independent per-fiber systems). */
fib_status fibers_create(const fib_params* p, int32_t n_fibers, const int32_t* n_nodes,
                         const int32_t* mu_of_fiber, const int32_t* junction_node, const float* vm0,
                         const fib_tuning* tuning, void* cuda_stream, fib_ctx** out);

/* Sets the MU firing trains (sec:stimulation_times_callbacks).
 *   n_mu          number of motor units; MU ids in mu_of_fiber must be < n_mu.
 *   offsets       [n_mu + 1] CSR offsets into fire_times_ms (offsets[0] = 0).
 *   fire_times_ms firing times in ms, ascending within each MU, >= 0.
 * Replaces any previous trains.  Before the first call no fiber is
 * stimulated.  Errors: FIB_EINVAL (unsorted, negative, bad offsets). */
fib_status set_stimulus_times(fib_ctx* ctx, int32_t n_mu, const int64_t* offsets,
                              const double* fire_times_ms);

/* Enqueues n_steps >= 0 Strang split steps (eq:monodomain_strang) for all
 * fibers.  Split step i covers t in [i dt_split, (i+1) dt_split); i counts
 * from 0 at creation (or the index given to fibers_write_state).  Returns
 * after enqueueing.  Errors: FIB_EINVAL (n_steps < 0), FIB_ECUDA. */
fib_status step(fib_ctx* ctx, int64_t n_steps);

/* Copies V (mV, float) of every node in ragged order into out.
 *   capacity       elements available in out (>= sum(n_nodes)).
 *   out_is_device  0: out is host memory; 1: device memory of the context's GPU.
 * Synchronises the context's stream.  Errors: FIB_EINVAL (capacity),
 * FIB_ENONFINITE (state has NaN/Inf; out is still written), FIB_ECUDA.
 * Thesis: the state subset copied back after a block of GPU steps
 * (section "Code Generation for GPUs"). */
fib_status read_vm(fib_ctx* ctx, float* out, size_t capacity, int32_t out_is_device);

/* Enqueues the same read of V into host memory without waiting, so that the
 * copy overlaps the steps enqueued after it (the thesis's copy of the state
 * subset after a block of GPU steps, section "Code Generation for GPUs",
 * taken off the critical path).
 *   out     host memory of >= sum(n_nodes) floats (capacity), ragged order.
 *           It must stay valid, and the caller must not read it, until
 *           read_vm_wait on the returned ticket returns.  Page-locked memory
 *           (cudaHostAlloc, a pinned torch tensor) lets the call return at
 *           once; with pageable memory it returns after the copy.
 *   ticket  (nullable) receives this read's number, 0, 1, 2, ... per context.
 * The values are V after the steps enqueued before the call.  A gather
 * kernel on the context's stream writes them into one of two device staging
 * buffers of the context (allocated, with a second stream, on the first
 * call); the copy to out runs on that second stream.  A third read in flight
 * makes the GPU, not the host, wait until the first read's copy is done.
 * Errors: FIB_EINVAL (capacity, out NULL), FIB_ENOMEM, FIB_ECUDA. */
fib_status read_vm_async(fib_ctx* ctx, float* out, size_t capacity, int64_t* ticket);

/* Waits until the read with this ticket has reached host memory.  Returns
 * the read's status: FIB_ENONFINITE if a value it read is NaN/Inf (out is
 * still written), or the step kernels' error (FIB_ETIMEOUT, FIB_ESTATE) as it
 * stood when the read was taken.  Reads share two staging buffers, so for a
 * ticket older than the two latest the status is that of the latest read
 * through the same buffer (errors persist, so none is lost).  Does not wait
 * for steps enqueued after the read.  fibers_synchronize and fibers_destroy
 * also wait for every read.  Errors: FIB_EINVAL (ticket never issued),
 * FIB_ECUDA.  Thesis: the end of the state copy of read_vm_async (section
 * "Code Generation for GPUs"). */
fib_status read_vm_wait(fib_ctx* ctx, int64_t ticket);

/* read_vm for callers that cannot allocate device memory.  The thesis has
 * no counterpart to this call; it exists for the library's users.  read_vm
 * with a host buffer stages V through device memory that the context
 * allocates with cudaMalloc on its first host read.  Some callers cannot
 * allow that: an application whose device memory is fully reserved by
 * another allocator (a framework's memory pool sized to the whole GPU) can
 * see that cudaMalloc fail with out-of-memory in the middle of a long run,
 * and a latency-sensitive loop cannot accept the device-wide
 * synchronisation that cudaMalloc and cudaFree may imply.  This call stages
 * through a fixed 8 MiB array compiled into the library instead (every GPU
 * that loads the library holds it until the process exits), and calls no
 * cudaMalloc, cudaFree or allocating routine.
 *   host_out  host buffer for V (mV, float, ragged order), capacity >= sum(n_nodes).
 * Limit: at most 2,097,152 nodes per context (the array's size); larger
 * contexts get FIB_EINVAL and should use read_vm.  The array's device
 * memory is reserved, and its device address looked up
 * (cudaGetSymbolAddress), by fibers_create on the context's GPU, so the
 * first read_vm_static call does not reserve it even under CUDA's lazy
 * module loading.  Only if that look-up failed at creation does the first
 * call on a GPU try again, and it may then reserve the array; make such a
 * call before any stream capture begins.  All calls share the array and it
 * keeps the last call's contents; calls that overlap on the GPU (two
 * contexts reading on different streams at once) race on it.  The calling
 * thread's current device is the same after the call as before it.
 * Synchronises the context's stream.  Errors as read_vm. */
fib_status read_vm_static(fib_ctx* ctx, float* host_out, size_t capacity);

/* Copies the full state into out (capacity >= 4 sum(n_nodes)): four blocks
 * of sum(n_nodes) floats in ragged order, u | dm | dh | dn, in the form the
 * library integrates: u = V - Vrest is the depolarisation in mV, and each HH
 * gate is held as its deviation from the resting value, dm = m - m0 and so
 * on, with (Vrest, m0, h0, n0) given by fibers_rest_state.  (In FP32 an
 * absolute gate near rest stops relaxing once a Heun increment falls below
 * half a unit in its last place; the deviation keeps full relative
 * precision, as u does for V.)  The copy is bit-exact, so it can serve as a
 * checkpoint.  Synchronises.  Same errors as read_vm.
 * Thesis: the state vector y = (V, m, h, n) of every model instance
 * (eq:subcellular); the thesis copies back only the subset needed for
 * output (section "Code Generation for GPUs") and has no checkpoint call. */
fib_status fibers_read_state(fib_ctx* ctx, float* out, size_t capacity, int32_t out_is_device);

/* Replaces the full state with in (layout of fibers_read_state: u | dm | dh
 * | dn) and sets the index of the next split step to step_index (>= 0).  Used
 * for checkpoint / resume: k steps, read_state, write_state, n - k steps
 * gives bit-for-bit the same state as n steps.  Clears a pending non-finite
 * flag, and in surrogate mode empties the network-node lists.  The thesis
 * has no counterpart (its initial state is sent to the GPU once, section
 * "Code Generation for GPUs"); this call exists for resuming runs.
 * Errors: FIB_EINVAL (count != 4 sum(n_nodes), step_index < 0), FIB_ECUDA. */
fib_status fibers_write_state(fib_ctx* ctx, const float* in, size_t count, int32_t in_is_device,
                              int64_t step_index);

/* Index of the next split step, and nodes handled by the fallback path in
 * surrogate mode (0 otherwise).  Synchronises.  No thesis counterpart (a
 * diagnostic of this library); errors as fibers_synchronize. */
fib_status fibers_stats(fib_ctx* ctx, int64_t* steps_done, int64_t* fallback_nodes);

/* Fiber-steps the adaptive scheme skipped so far (0 without
 * FIB_FLAG_ADAPTIVE).  Synchronises.  Thesis: the points in equilibrium
 * that adaptive computation leaves out (sec:adaptive_computation_for_fiber_based). */
fib_status fibers_adaptive_stats(fib_ctx* ctx, int64_t* skipped_fiber_steps);

/* Waits for all enqueued work and reports device-side errors: FIB_ENONFINITE
 * (state became NaN/Inf), FIB_ESTATE (surrogate node list overflowed),
 * FIB_ETIMEOUT (with split warp roles, a bounded wait between the reaction
 * and diffusion warps gave up; the state is unreliable), FIB_ECUDA.  Also
 * waits for every read_vm_async.  Thesis: the point of synchronisation between blocks of GPU
 * timesteps (section "Code Generation for GPUs"). */
fib_status fibers_synchronize(fib_ctx* ctx);

/* Reads / changes the launch shape.  Changing it keeps the state.  The
 * thesis has no counterpart: it distributes whole fibers to processes for
 * load balance (sec:partitioning_requirements), while here fibers are packed
 * into thread blocks by the layout these values choose.  Errors: FIB_EINVAL
 * (a value out of range, fibers too long for the shape; the old shape stays),
 * FIB_ENOMEM, FIB_ECUDA. */
fib_status fibers_get_tuning(const fib_ctx* ctx, fib_tuning* out);
fib_status fibers_set_tuning(fib_ctx* ctx, const fib_tuning* tuning);

/* Times candidate launch shapes on this context's own fibers for n_trial_steps
 * split steps each, keeps the fastest, and restores the state, step index and
 * adaptive skip count so the simulation is unchanged.  best (nullable)
 * receives the choice.  Synchronises.  No thesis counterpart (see
 * fibers_set_tuning).  Errors: FIB_EINVAL (n_trial_steps < 1), FIB_ENOTSUP
 * (surrogate mode, whose step kernel it does not time), FIB_ECUDA.
 *
 * The choice is cached for the process, keyed by the GPU model (name, SM
 * count, compute capability), the mode, flags, splitting and diffusion
 * scheme, r = c dt_1D / h^2, the substep counts and the length histogram
 * (every distinct fiber length with its number of fibers).  A later call on
 * a context with an equal key applies the cached shape (like
 * fibers_set_tuning, keeping the context's steps_per_launch and graph_steps)
 * and launches no trial steps. */
fib_status fibers_autotune(fib_ctx* ctx, int32_t n_trial_steps, fib_tuning* best);

/* The autotune cache.  size: entries held.  clear: drops them all.  save:
 * writes every entry to a text file (first line "fibers-autotune-cache 1",
 * then one line per entry; the layout is described in the implementation).
 * load: merges a file's entries into the cache (an entry with an equal key
 * is replaced); nothing is merged unless every line parses.  Host-only, no
 * thesis counterpart.  Errors: FIB_EINVAL (NULL path, malformed file; the
 * message names the line), FIB_EIO (file cannot be opened, read or
 * written); the message is read with fibers_last_error(NULL). */
int64_t fibers_autotune_cache_size(void);
fib_status fibers_autotune_cache_clear(void);
fib_status fibers_autotune_cache_save(const char* path);
fib_status fibers_autotune_cache_load(const char* path);

/* ---------------------------------------------------------------------------
 * Reaction-step surrogate (FIB_MODE_SURROGATE).
 *
 * A small network replaces the reaction part of each split step (the Heun
 * substeps of the HH model, eq:heun, sec:subcelullar_model); the diffusion
 * halves stay exact.  The thesis has no learned component on this path.
 * Network: x = normalised (u, m, h, n, s) -> 128 -> SiLU -> 128 -> SiLU -> 4
 * outputs, the normalised change of (u, m, h, n) over one split step, where
 * u = V - Vrest and s is the fraction of the step's Heun substeps with the
 * stimulus on.  SiLU(z) = z / (1 + exp(-z)).  Inference runs on BF16 tensor
 * cores with FP32 accumulation; every input is split into bf16 high and low
 * parts so the first layer sees it to FP32 accuracy.  A node whose input lies
 * outside the training envelope is advanced by the plain HH step instead.
 *
 * Parameter vector theta (FP32, kNumParams = 17796 values): W1 (128 x 5,
 * row-major), b1 (128), W2 (128 x 128), b2 (128), W3 (4 x 128), b3 (4).
 * ------------------------------------------------------------------------- */

/* Loads a trained surrogate into a context created with FIB_MODE_SURROGATE.
 *   blob      host array of n_floats = 17837 floats: 5, 128, 4, then
 *             in_mu[5], in_sigma[5] (x = (raw - in_mu) / in_sigma),
 *             out_mu[4], out_sigma[4] (change = out * out_sigma + out_mu),
 *             env_lo[5], env_hi[5] (raw inputs outside [lo, hi] use the
 *             plain HH step), quiet_lo[5], quiet_hi[5] (raw inputs inside
 *             this box around rest also use the plain HH step, which keeps
 *             rest an exact fixed point), theta[17796].
 * raw = (u, m, h, n, s). 
 * Copied; the caller keeps the blob.  Errors: FIB_EINVAL (size, shape,
 * non-finite values, in_sigma <= 0), FIB_ESTATE (not a surrogate context).
 * No thesis counterpart: the surrogate is this library's addition (see the
 * section comment above). */
fib_status fibers_load_surrogate(fib_ctx* ctx, const float* blob, size_t n_floats);

/* The plain reaction step (dt_split / dt_0d Heun substeps of the HH model,
 * eq:heun) on `count` independent nodes, for generating training targets.
 *   in        device, 4 x count floats: V (mV) | m | h | n.
 *   stim_mask device, count bytes (bit k: stimulus on during substep k), or NULL.
 *   out       device, 4 x count floats, same layout as in.
 * Asynchronous on cuda_stream.  Errors: FIB_EINVAL, FIB_ECUDA. */
fib_status fibers_hh_reaction(const fib_params* p, int64_t count, const float* in, const uint8_t* stim_mask,
                              float* out, void* cuda_stream);

/* One training step of the surrogate network on a batch (device buffers):
 * forward pass, mean-squared-error loss over the batch and the 4 outputs, and
 * the gradient of the loss with respect to theta.  With quantize != 0 the
 * forward pass rounds weights and matrix-product inputs to bfloat16 (round to
 * nearest even) as inference does, and the gradient treats that rounding as
 * the identity; every matrix product (forward, backward and the weight
 * gradients) then runs on BF16 tensor cores with FP32 accumulation, with
 * FP32 left operands split into bf16 high and low parts.  With quantize == 0
 * the kernels compute in FP32 on the CUDA cores.  Deterministic (no atomics).
 *   theta     17796 floats.      x       batch x 5 normalised inputs.
 *   target    batch x 4.         workspace >= batch x 848 floats (scratch).
 *   grad      17796 floats (out). loss   1 float (out, device).
 * Asynchronous.  Errors: FIB_EINVAL, FIB_ECUDA.  No thesis counterpart
 * (training of the surrogate network). */
fib_status fibers_mlp_train_step(const float* theta, int32_t quantize, const float* x, const float* target,
                                 int64_t batch, float* workspace, float* grad, float* loss, void* cuda_stream);

/* Forward pass only: out (batch x 4) for inputs x (batch x 5); workspace >=
 * batch x 520 floats.  Asynchronous.  Errors: FIB_EINVAL, FIB_ECUDA.  No
 * thesis counterpart (the surrogate network). */
fib_status fibers_mlp_forward(const float* theta, int32_t quantize, const float* x, int64_t batch, float* workspace,
                              float* out, void* cuda_stream);

/* One Adam update of n parameters in place (Kingma & Ba 2015, with bias
 * correction for step t >= 1).  All buffers on the device.
 *   theta_avg  NULL, or n floats updated after the step to the exponential
 *              moving average of the weights (Polyak averaging in its
 *              exponential form): theta_avg = avg_decay * theta_avg +
 *              (1 - avg_decay) * theta.  The caller initialises it (for
 *              example with theta before the first step).
 *   avg_decay  in [0, 1]; ignored when theta_avg is NULL.
 * Asynchronous.  Errors: FIB_EINVAL (n < 1, t < 1, a NULL buffer, avg_decay
 * outside [0, 1]), FIB_ECUDA.  No thesis counterpart (surrogate training). */
fib_status fibers_adam_step(float* theta, float* m, float* v, const float* grad, int64_t n, float lr, float beta1,
                            float beta2, float eps, int64_t t, float* theta_avg, float avg_decay, void* cuda_stream);

/* Per-column mean, standard deviation, minimum and maximum of a device matrix
 * X (n x cols, row-major) into out (host, 4 x cols doubles, column by column:
 * mean, std, min, max).  Synchronises cuda_stream.  cols <= 64.  Errors:
 * FIB_EINVAL, FIB_ECUDA.  No thesis counterpart (input normalisation of the
 * surrogate network). */
fib_status fibers_feature_stats(const float* X, int64_t n, int32_t cols, double* out, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Coupling to a 3D mesh of the muscle (eq:discretized_fibers): the
 * transmembrane voltage of the fibers is mapped onto a structured
 * hexahedral mesh (eq:discretized_fibers_2) and the static first bidomain
 * equation gives the extracellular potential (eq:discretized_fibers_3,
 * eq:static_bidomain_rhs):
 *     K_(sigma_i + sigma_e) phi_e = -K_(sigma_i) V3D
 * with trilinear finite elements on the mesh, homogeneous Neumann
 * boundaries (eq:monodomain_bc3), sigma_i = sigma_i a (x) a along the fiber
 * direction a = z and sigma_e isotropic (eq:multidomain_isotropic_e).
 * The mapping is the thesis's data mapping between meshes
 * (sec:data_mapping_between_meshes, eq:mapping_source_target): each fiber
 * node adds the value of its element's 8 trilinear ansatz functions at its
 * position as factors to those nodes, and a 3D node's value is the
 * factor-weighted mean of the fiber nodes that reach it (0 if none does).
 * The Neumann problem fixes phi_e up to a constant; the library returns the
 * solution with zero mean over the 3D nodes.
 * ------------------------------------------------------------------------- */

typedef struct fib_emg fib_emg;

/* Structured 3D mesh: node (i, j, k) at origin + (i, j, k) * spacing, node
 * index i + nx (j + ny k).  Units cm and mS/cm. */
typedef struct {
  int32_t nx, ny, nz;  /* nodes per direction, each >= 2 */
  int32_t reserved;    /* must be 0 */
  double origin[3];
  double spacing[3];   /* > 0 */
  double sigma_i;      /* intracellular conductivity along the fibers (>= 0), e.g. 8.93 */
  double sigma_e;      /* extracellular conductivity, isotropic (> 0), e.g. 6.7 */
} fib_mesh3d;

/* Builds the mapping from the fibers of ctx to the 3D mesh.  Fibers are
 * straight lines along z: fiber f at (fiber_xy[2f], fiber_xy[2f+1]), its
 * node i at z = z0 + i h (h of fib_params).  Points outside the mesh are
 * clamped onto its boundary elements.  ctx must outlive the returned
 * object, which owns its device memory (mapping in CSR form, about 8 x 8
 * bytes per fiber node).  Synchronises.  Errors: FIB_EINVAL (sizes,
 * spacing, conductivities, non-finite positions; message on ctx),
 * FIB_ENOMEM, FIB_ECUDA, FIB_ENOTSUP (no cooperative launch).  Thesis:
 * sec:data_mapping_between_meshes, eq:mapping_source_target. */
fib_status fibers_emg_create(fib_ctx* ctx, const double* fiber_xy, double z0, const fib_mesh3d* mesh,
                             fib_emg** out);

/* V3D (mV, FP64) of every 3D node for the fibers' current V, into out
 * (capacity >= nx ny nz; out_is_device selects device or host memory).
 * Synchronises.  Errors: FIB_EINVAL, FIB_ECUDA (message:
 * fibers_emg_last_error).  Thesis: eq:discretized_fibers_2 (the prolongation
 * of V onto the 3D mesh). */
fib_status fibers_emg_vm3d(fib_emg* emg, double* out, size_t capacity, int32_t out_is_device);

/* phi_e (mV, written as float) of every 3D node for the fibers' current V:
 * the mapping, the right-hand side and a Jacobi-preconditioned conjugate
 * gradient solve in FP64, stopped once the residual is below rtol times
 * the right-hand side's norm, or after max_iter iterations.  iterations and
 * rel_residual (nullable) receive what the solve reached.  Synchronises.
 * Errors: FIB_EINVAL, FIB_ECUDA, FIB_ETIMEOUT (rtol not reached; out holds
 * the last iterate).  Thesis: eq:discretized_fibers_3, eq:static_bidomain_rhs. */
fib_status fibers_emg_phi_e(fib_emg* emg, float* out, size_t capacity, int32_t out_is_device, double rtol,
                            int32_t max_iter, int32_t* iterations, double* rel_residual);

/* Number of 3D nodes (0 for NULL).  No thesis counterpart. */
int64_t fibers_emg_nodes(const fib_emg* emg);

/* Message of the last failing call on emg (never NULL).  No thesis
 * counterpart. */
const char* fibers_emg_last_error(const fib_emg* emg);

/* Frees the mapping and solver memory.  NULL is allowed.  No thesis
 * counterpart. */
void fibers_emg_destroy(fib_emg* emg);

/* Host-only diagnostic (no GPU needed): the coefficient tables of the
 * partitioned tridiagonal solve that fibers_create builds for a fiber of
 * n_nodes nodes at K nodes per thread, for the Crank-Nicolson matrix of
 * eq:lumping_crank_nicolson_2 with r = c dt_1d / h^2 (rows (1+r, -r),
 * (-r/2, 1+r, -r/2), (-r, 1+r)).
 *   fp64_solve  0: the FP32 solve's PCR cutoff (2^-32); 1: the FP64 one (2^-40).
 *   levels      out: PCR levels kept.   threads  out: threads per fiber (Tw).
 *   rows        NULL, or 2 x K x 5 doubles: the interior chunk's row
 *               coefficients, then the fiber's last chunk's; per row
 *               (F1, F2, G, Ap, Bt) of the chunk elimination.
 *   recs        NULL, or threads x (7 + 3 levels) doubles: per thread
 *               (1/B, A/B, C/B, c0, KE, KD, KDn) of the reduced system, then
 *               (1/b, a/b, c/b) per PCR level.
 * Call with NULL tables first to learn levels and threads.  Errors:
 * FIB_EINVAL (K not 4, 8, 12 or 16; n_nodes < 1 or more than 256 K; r < 0
 * or not finite; a zero pivot). */
fib_status fibers_solver_tables(int32_t K, double r, int32_t n_nodes, int32_t fp64_solve, int32_t* levels,
                                int32_t* threads, double* rows, double* recs);

/* The resting state the library uses for parameters p (host only, no
 * GPU): out[0] = Vrest, out[1..3] = the steady-state gates m0, h0, n0 of
 * the HH rates at Vrest (sec:subcelullar_model; exp* rates with
 * FIB_FLAG_EXP_APPROX), as floats.  fibers_read_state's gate blocks are
 * deviations from these values.  Errors: FIB_EINVAL (invalid parameters or
 * out NULL). */
fib_status fibers_rest_state(const fib_params* p, float* out);

/* Number of launches of this library's kernels enqueued so far by ctx (a
 * diagnostic of this library, no thesis counterpart; 0 for ctx == NULL). */
int64_t fibers_kernel_launches(const fib_ctx* ctx);

/* Message of the last failing call on ctx (never NULL).  With ctx == NULL:
 * the message of the last failed call on this thread that had no context
 * (fibers_create, the autotune cache calls).  No thesis counterpart. */
const char* fibers_last_error(const fib_ctx* ctx);

/* Frees everything the context owns, after waiting for its stream.  NULL is
 * allowed.  No thesis counterpart. */
void fibers_destroy(fib_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FIBERS_H_ */
