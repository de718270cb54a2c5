/*
 * ttn_heom.h -- C ABI of the GB300 (sm_103a) TTN-HEOM propagation library.
 *
 * The library propagates the extended density operator (EDO) of the bexcitonic
 * HEOM (TENSO paper, Sec. 2.2, Eq. heom-std) stored as a tree tensor network
 * (Sec. 2.3, Eq. omega_tensor) under a sum-of-products (SOP) generator
 * (Eq. master_lvn), with the fixed-rank (ps1) and adaptive-rank (ps2)
 * projector-splitting integrators (Sec. 2.3, last paragraph), and returns the
 * reduced density matrix rho_S = <0|Omega> (Sec. 2.2).
 *
 * Conventions shared by every entry point
 *  - Complex numbers are two consecutive doubles (real, imaginary).
 *  - Matrices are row-major. An operator acting on a leg of dimension d is a
 *    d x d matrix M that maps amplitude index a to a': new[a'] = sum_a M[a'][a] old[a].
 *  - Legs: leg 0 = system ket index i, leg 1 = system bra index j, legs 2.. =
 *    Fock legs of the bath features (Eq. EDO-elements). Legs 0 and 1 must sit
 *    on the root node 0. A right multiplication B A^dagger of the system density
 *    matrix acts on leg 1 with the matrix conj(A) (Sec. 2.2, A^< B = B A^dagger).
 *  - Node tensors are stored row-major with their legs in canonical order:
 *    the parent bond first (absent at the root), then the child nodes and
 *    open legs sorted by the smallest open-leg index below them. Only nodes
 *    with exactly three legs are supported (tensor trains and binary trees).
 *  - Ownership: every host array passed in is read during the call and never
 *    retained. Device memory is one caller-provided workspace (see
 *    ttn_workspace_size / ttn_set_workspace); the library allocates no device
 *    memory itself. The caller frees the workspace after ttn_destroy.
 *  - Errors: every entry point returns a ttn_status and never aborts;
 *    ttn_last_error(h) describes the last failure. A failing call leaves the
 *    handle in the state it had before the call, except that TTN_ECUDA from
 *    any call, and TTN_ENUMERIC / TTN_ETIMEOUT from ps1 steps (which run
 *    asynchronously and report a failure at a later synchronising call),
 *    leave the state undefined (re-seed with ttn_set_rdo0 or ttn_set_node).
 *    ps2, vmf and mix steps run under host control: one that fails with
 *    TTN_ETIMEOUT or TTN_ENUMERIC puts back the time, ranks and node tensors
 *    the handle had at the start of the call.
 *  - A handle is not thread safe; distinct handles are independent.
 *  - All device work is issued on the stream given by ttn_set_stream
 *    (default: the legacy default stream). Calls that return host data
 *    (ttn_rdm, ttn_get_node) synchronise that stream.
 */
#ifndef TTN_HEOM_H
#define TTN_HEOM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ttn_ctx* ttn_t;

typedef enum {
  TTN_OK = 0,
  TTN_EINVAL = 1,        /* bad argument (tree, dims, ranks, operator, size) */
  TTN_ENOMEM = 2,        /* workspace too small or not set */
  TTN_ECUDA = 3,         /* a CUDA call failed (message in ttn_last_error) */
  TTN_ENUMERIC = 4,      /* non-finite value detected in the state */
  TTN_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
  TTN_ESTATE = 6,        /* call out of order (e.g. ttn_step before sop_load) */
  TTN_EUNSUPPORTED = 7   /* valid request the library does not implement */
} ttn_status;

/* Arithmetic of the node and bond contractions. QR, SVD, RK4 stage
 * accumulation and the reduced density matrix are FP64 in every mode. */
enum { TTN_FP64 = 0, TTN_MIXED_FP32 = 1 };

/* Propagation schemes (Sec. 2.3, Sec. 7.5): ps1 fixed rank, ps2 adaptive rank,
 * vmf direct integration of all node equations at fixed rank (FP64 form),
 * mix = ps2 until a bond rank reaches max_rank, vmf from then on (the
 * paper's default strategy). */
enum { TTN_PS1 = 1, TTN_PS2 = 2, TTN_VMF = 3, TTN_MIX = 4 };

/* Tree topology: parent[0] = -1 (node 0 is the root), parent[u] in [0, n_nodes)
 * otherwise; leg_node[l] = node carrying open leg l. */
typedef struct {
  int32_t n_nodes;
  const int32_t* parent;
  int32_t n_legs;
  const int32_t* leg_node;
} ttn_tree;

/* Numerical parameters (defaults in parentheses).
 *  qr_tol    (1e-9)  Householder QR treats a column whose remaining norm is at
 *                    most qr_tol*||A||_F as exactly dependent: no reflector,
 *                    R_jj = 0, Q column = H_0..H_{j-1} e_j. Much smaller
 *                    values let rounding decide the completion of nearly
 *                    dependent columns, and long fixed-rank trajectories then
 *                    depend on the order of the sums.
 *  kappa     (2.5)   RK4 substeps per flow of length tau:
 *                    m = max(1, ceil(|tau| * Lambda / kappa - 1e-9)), Lambda =
 *                    sum over terms of |coef| * prod ||op||_2 (|coef| * g_bound
 *                    for driven terms), fixed at sop_load.
 *  ps2_atol  (1e-7)  ps2 keeps r0 = #{sigma > ps2_atol} ... (Sec. 4, Table 4)
 *  ps2_ratio (2)     ... and then min(cap, max(1, ceil(ps2_ratio * r0))) values.
 *  max_rank  (32)    ps2 bond-rank cap (Sec. 4, Table 4: max_auxiliary_rank).
 *  svd_tol   (1e-12) kept singular values <= svd_tol*sigma_1 are replaced by a
 *                    deterministic completion with zero weight.
 *  max_split (16)    1..16: at most this many CTAs (one thread-block cluster)
 *                    share one output tile of a contraction launch; launches
 *                    smaller than two CTAs per SM are split up to this factor
 *                    (no counterpart in the paper: GB300 work distribution).
 *                    Use 1 for instances advanced concurrently by
 *                    ttn_batch_step, which fill the GPU by themselves.
 *  tensor_cores (1)  mixed form only: run the mode products of large nodes
 *                    (contracted legs <= 64, >= 16384 elements) on the
 *                    tcgen05 tensor cores in 3xTF32 (hi/lo split, FP32
 *                    accumulation); 0 keeps them on the FP32 CUDA cores.
 *                    1 stages the tensor operand by the threads, chunk by
 *                    chunk; 2 splits the tensor operands into tf32 hi / lo
 *                    tiles first and streams both operands by bulk copies
 *                    through a 4-stage ring (one producer thread, one MMA
 *                    thread). Both give the same results bit for bit; on the
 *                    rank-64 chain the ring kernel is ~15 % faster per launch
 *                    but its split pass costs as much as it saves.
 *  wait_s    (2.0)   0..60: upper bound, in seconds, of the device-side waits
 *                    of the kernels whose blocks wait on one another through
 *                    global memory (the grid barriers of the Jacobi SVD and of
 *                    the blocked QR's panels over the whole GPU); a wait that
 *                    runs out is reported as TTN_ETIMEOUT by the next
 *                    synchronising call (a ps2 / mix step puts its state
 *                    back, a ps1 step leaves it undefined; no counterpart in
 *                    the paper). The cluster QR's exchanges keep a fixed 2 s
 *                    bound.
 *  ode_rtol  (1e-5)  vmf: relative and absolute tolerance of the dopri5
 *  ode_atol  (1e-7)  controller (Sec. 4, Table 4 defaults).
 *  vmf_atol  (1e-10) vmf: added to the diagonal of every single-hole density
 *                    matrix before it is inverted (Sec. 7.5 regularisation).
 *  tile_warps (0)    0, 2, 4 or 8: warps per CTA sharing one 32-output tile of
 *                    the CUDA-core contraction launches (0: 8). Setting it (or
 *                    max_split) replaces the launch shapes of every job list
 *                    by the planned ones; ttn_autotune then picks warps and
 *                    split per list. Fewer warps per tile waste less on idle
 *                    warps and reductions when many instances run at once
 *                    (no counterpart in the paper). */
typedef struct {
  double qr_tol;
  double kappa;
  double ps2_atol;
  double ps2_ratio;
  int32_t max_rank;
  double svd_tol;
  int32_t max_split;
  int32_t tensor_cores;
  double wait_s;
  double ode_rtol;
  double ode_atol;
  double vmf_atol;
  int32_t tile_warps;
} ttn_params;

/* Create a handle (Sec. 2.3, Eq. omega_tensor). leg_dims[n_legs]: leg
 * dimensions (leg 0 and 1 both M). ranks[n_nodes]: requested rank of the bond
 * between node u and its parent (ranks[0] ignored); each is capped to the
 * product of the other leg dimensions at either end node, iterated to a fixed
 * point (ttn_get_ranks reports the result). precision: TTN_FP64 or
 * TTN_MIXED_FP32. Returns TTN_EINVAL for a parent array that is not a tree
 * rooted at 0, legs 0/1 not on the root, a node without three legs, dims < 1,
 * ranks < 1. Host-only: no device work. */
ttn_status ttn_create(const ttn_tree* tree, const int32_t* leg_dims, const int32_t* ranks,
                      int32_t precision, ttn_t* out);

/* Set numerical parameters; may be called any time before ttn_set_workspace
 * (max_rank changes the workspace size for ps2). */
ttn_status ttn_set_params(ttn_t h, const ttn_params* p);
ttn_status ttn_get_params(ttn_t h, ttn_params* p);

/* Load the SOP generator of Eq. master_lvn:
 *     L(t) = sum_m coef_m * g_{d_m}(t) * prod_{f in term m} op_f on leg(op_f).
 * Local operators: op k acts on leg op_leg[k] with d = leg_dims[op_leg[k]]; its
 * d*d complex entries start at op_data[2*op_offset[k]] (offsets in complex
 * elements). Terms: term m uses ops term_ops[term_offsets[m] .. term_offsets[m+1]-1]
 * (at most two, on distinct legs); coef[2m], coef[2m+1] its complex
 * coefficient; coef_drive[m] = -1 (static) or a drive id >= 0 whose g(t)
 * multiplies the coefficient (driven terms may only act on legs of the root).
 * Terms are merged on the host into per-bond operator classes (single-leg sums
 * and two-leg groups keyed by their more shared factor). Host-only.
 * Errors: TTN_EINVAL (bad leg, dims, op id, more than two factors, repeated
 * leg in one term, non-finite entry), TTN_EUNSUPPORTED (driven term off the root). */
ttn_status sop_load(ttn_t h, int32_t n_ops, const int32_t* op_leg, const int64_t* op_offset,
                    const double* op_data, int32_t n_terms, const int32_t* term_offsets,
                    const int32_t* term_ops, const double* coef, const int32_t* coef_drive);

/* Drive d: g(t, user) is sampled on the host at the half-step midpoints
 * t0 + dt/4 and t0 + 3dt/4 of every step (the driven system term is frozen
 * during each half sweep); g_bound >= max |g| enters Lambda. Must precede
 * ttn_set_workspace. */
typedef double (*ttn_drive_fn)(double t, void* user);
ttn_status ttn_set_drive(ttn_t h, int32_t id, ttn_drive_fn g, void* user, double g_bound);

/* Device workspace: bytes needed for the state, environments, operators and
 * scratch (sized for the rank caps). Valid after sop_load. */
ttn_status ttn_workspace_size(ttn_t h, size_t* bytes);
/* Bind a device buffer of at least ttn_workspace_size bytes, 256-byte aligned,
 * on the current CUDA device. Uploads operators, builds the initial product
 * state rho0 = |0><0| (x) |0..0> and its environments. */
ttn_status ttn_set_workspace(ttn_t h, void* device_ptr, size_t bytes);
/* cudaStream_t passed as void*. */
ttn_status ttn_set_stream(ttn_t h, void* stream);

/* Initial product state Omega(0) = rho0 (x) |0..0> (Sec. 2.2): root
 * A[i,j,0] = rho0[i][j], other root entries 0; every other core
 * U[a, flat(children)] = delta(a, flat) (the first r columns of the identity).
 * rho0: M*M complex, row-major. Resets time to 0 and rebuilds environments. */
ttn_status ttn_set_rdo0(ttn_t h, const double* rho0);

/* Advance n_steps steps of length dt. TTN_PS1 / TTN_PS2: one step = the
 * symmetric composition of a half sweep over dt/2 and its adjoint. TTN_VMF:
 * every node tensor advanced together over dt by the Dormand-Prince 5(4) pair
 * with adaptive substeps (ode_rtol, ode_atol; the trial step carried from one
 * call to the next) under the multilayer-MCTDH node equations -- the root
 * carries the weight, every other node stays semi-unitary (its derivative is
 * projected off its own span) and is multiplied by the inverse of its
 * regularised single-hole density matrix (vmf_atol); FP64 form only
 * (TTN_EUNSUPPORTED in the mixed form); not captured as a graph (the step
 * control synchronises). TTN_MIX: ps2 steps until a bond reaches max_rank,
 * TTN_VMF steps at the reached ranks afterwards (reset by ttn_set_rdo0). The
 * orthogonality centre is at the root before and after. Asynchronous on the
 * handle's stream except for drive sampling on the host. For an autonomous
 * generator on a non-default stream the kernels of one ps1 step are captured
 * once as a CUDA graph (per dt) and replayed. A non-finite amplitude is
 * detected on the device once per call and reported as TTN_ENUMERIC by the
 * next synchronising call (ttn_rdm, ttn_get_node). Kernels whose blocks wait on
 * one another (the QR of a cluster of CTAs; the panels of the blocked QR of
 * matricisations taller than a cluster holds, a cooperative launch of one
 * CTA per SM) bound every wait to a few seconds; a wait that gives up is
 * reported as TTN_ETIMEOUT by the next synchronising call. */
ttn_status ttn_step(ttn_t h, double dt, int32_t scheme, int32_t n_steps);

/* rho_S = <0|Omega>: contract every feature leg with the n = 0 vector.
 * rho_out: caller-allocated host buffer of M*M complex, row-major. Synchronises. */
ttn_status ttn_rdm(ttn_t h, double* rho_out);
/* Same, written asynchronously to a device buffer of M*M complex. */
ttn_status ttn_rdm_device(ttn_t h, void* rho_dev);

/* Effective bond ranks (ranks_out[n_nodes], entry 0 = 0); for ps2 the current ones. */
ttn_status ttn_get_ranks(ttn_t h, int32_t* ranks_out);
/* Current dims of node u's three legs in canonical order. */
ttn_status ttn_node_shape(ttn_t h, int32_t u, int32_t* dims3);
/* Copy node tensor u (prod(dims) complex) to / from the host. ttn_set_node
 * requires non-root nodes to be semi-unitary toward their parent (Eq.
 * semiunitary); environments are rebuilt before the next step. Synchronises. */
ttn_status ttn_get_node(ttn_t h, int32_t u, double* host_out);
ttn_status ttn_set_node(ttn_t h, int32_t u, const double* host_in);
/* Simulation time reached (starts at 0, Sec. 7.1 checkpoint convention). */
ttn_status ttn_time(ttn_t h, double* t);
/* Checkpoint (Sec. 7.1, checkpoint files): the whole propagated state of a
 * handle -- simulation time, current bond ranks and every node tensor (FP64,
 * canonical layout) -- as one self-describing byte blob, with the tree, the
 * leg dimensions and a fingerprint (FNV-1a) of the loaded generator
 * (operators, terms, drives) that a loading handle must match; the paper
 * likewise requires the loading run to use the same Hamiltonian, operators,
 * baths, depth and ranks. Unlike the paper's files, which restart the clock
 * at zero, the blob keeps the time (drives depend on it).
 * ttn_checkpoint_size: bytes of a blob of the current state.
 * ttn_checkpoint_save: writes it to a caller-allocated host buffer of at least
 *   that size; synchronises.
 * ttn_checkpoint_load: restores a blob into a bound handle built for the same
 *   model (ranks may differ from the handle's current ones, e.g. after ps2,
 *   but not exceed its capacities); environments are rebuilt, the captured
 *   step graph dropped. The learned rank proposer's per-bond history is not
 *   part of the blob. Errors: TTN_EINVAL (not a checkpoint, other topology,
 *   dims or generator, rank beyond capacity, truncated, non-finite),
 *   TTN_ESTATE (no workspace). A failing load leaves the state undefined only
 *   after the rank check (re-seed with ttn_set_rdo0). */
ttn_status ttn_checkpoint_size(ttn_t h, size_t* bytes);
ttn_status ttn_checkpoint_save(ttn_t h, void* host_buf, size_t bytes);
ttn_status ttn_checkpoint_load(ttn_t h, const void* host_buf, size_t bytes);

/* RK4 substeps used for a flow of length tau under the current generator. */
ttn_status ttn_substeps(ttn_t h, double tau, int32_t* m);

/* Propagate several independent handles (same scheme and dt) in one call.
 * With ps1 and autonomous generators on non-default streams, every handle's
 * captured step graph becomes one concurrent branch of a parent CUDA graph,
 * launched n_steps times on the first handle's stream; the other handles'
 * streams are ordered before and after the batch with events, so later calls
 * on any member see the result. The parent graph is cached in the first handle
 * and rebuilt when the member list, dt or a member's step graph changes.
 * Otherwise (drives, default streams, profiling) the handles are stepped one
 * after another. Every handle needs its own workspace. */
ttn_status ttn_batch_step(ttn_t* hs, int32_t n, double dt, int32_t scheme, int32_t n_steps);

/* Kernel accounting (instrumentation, not on the physics path). Kernel
 * classes: 0 = node/bond application (sum of mode products with the fused RK4
 * stage update), 1 = environment update (mode products + projection),
 * 2 = Householder QR, 3 = everything else (absorb, copies, RDM, drive, checks).
 * ttn_stats: launches and algorithmic FLOPs issued since the last reset
 * (complex multiply-add = 8 FLOPs), counted on the host, always on. Kind 4
 * (launches only) counts the job lists issued on the tensor-core ring path
 * (tensor_cores = 2), at issue time: a captured step graph counts once.
 * ttn_profile(h, 1) additionally brackets every launch with CUDA events on the
 * handle's stream (the step is then issued launch by launch, not as a graph);
 * ttn_profile(h, 2) keeps the captured step graph and records the bracketing
 * events as event-record nodes inside it, so the times are those of the
 * graph-replayed step (ttn_step then synchronises after every replay to read
 * them; launches outside a graph are bracketed as in mode 1). 0 turns it off.
 * ttn_profile_read synchronises and returns the summed device time of each
 * class in milliseconds. ttn_stats_reset clears both. */
ttn_status ttn_stats(ttn_t h, int32_t kind, int64_t* launches, double* flops);
ttn_status ttn_profile(ttn_t h, int32_t on);
ttn_status ttn_profile_read(ttn_t h, int32_t kind, double* ms);
ttn_status ttn_stats_reset(ttn_t h);

/* Learned rank proposer (not in the paper). A fixed 24-64-64-13 MLP (ReLU,
 * softmax over rank changes -4..+8) proposes, for every ps2 split, the new rank
 * of the bond from the bond's history (features below); the split is then
 * computed by a randomised range finder (Gaussian sketch of r + 8 columns,
 * Householder QR, Jacobi SVD of the small projected matrix). The proposal is
 * accepted only if the truncation rule applied to the sketch's singular values
 * cuts inside the sketch and the exact discarded weight
 * ||Theta||_F^2 - sum_{i<r} sigma_i^2 is at most ps2_atol^2; otherwise the full
 * Jacobi SVD rule runs. Features (24 floats): log10 of the bond's last
 * normalised singular values (16, /16, -1 if absent), rank / cap, log10 of the
 * last 4 discarded weights (/20, -1 if absent), log10(ps2_atol)/10,
 * ps2_ratio/4, 1. Parameters: one float vector (ttn_mlp_n_params entries) in
 * the order W1, b1, W2, b2, W3, b3, matrices row-major (output index first).
 *
 * ttn_mlp_forward: logits[batch*13] for x[batch*24]; ws: ttn_mlp_workspace_size bytes.
 * ttn_mlp_grad: mean softmax cross-entropy *loss (device float) and its gradient
 *   grads[n_params] for integer labels in 0..12; deterministic (fixed-order sums).
 * ttn_mlp_adam: one Adam step (beta 0.9/0.999, eps 1e-8, bias-corrected, t >= 1).
 * All pointers are device pointers; work is issued on `stream`.
 * ttn_split_log: the handle's log of full-SVD ps2 splits (features and the class
 *   clamp(r_rule - r_before, -4, 8) + 4 the truncation rule chose); copies up to
 *   max records to host arrays and returns the total in *n_total.
 * ttn_set_rank_proposer: device parameters the handle reads at every ps2 split
 *   (the caller keeps them alive; NULL turns the proposer off).
 * ttn_proposer_stats: splits that consulted the network and proposals accepted. */
ttn_status ttn_mlp_n_params(int32_t* n);
ttn_status ttn_mlp_workspace_size(int32_t batch, size_t* bytes);
ttn_status ttn_mlp_forward(const float* params, const float* x, int32_t batch, float* logits, void* ws,
                           void* stream);
ttn_status ttn_mlp_grad(const float* params, const float* x, const int32_t* labels, int32_t batch, float* grads,
                        float* loss, void* ws, void* stream);
ttn_status ttn_mlp_adam(float* params, float* m, float* v, const float* grads, int32_t t, float lr, void* stream);
ttn_status ttn_split_log(ttn_t h, float* feats, int32_t* labels, int32_t max, int32_t* n_total);
ttn_status ttn_split_log_clear(ttn_t h);
ttn_status ttn_set_rank_proposer(ttn_t h, const float* params_dev);
ttn_status ttn_proposer_stats(ttn_t h, int64_t* proposed, int64_t* accepted);

/* No-allocation RDM. The paper has no counterpart to this entry point; it is
 * a deployment aid. Some callers cannot allocate device memory at all: code
 * running inside another framework's memory pool or arena, or runtimes that
 * forbid allocation once they have started. Such a caller cannot give a handle
 * its workspace, so this call takes node tensors the caller already holds in
 * device memory and computes rho_S = <0|Omega> into rho_dev (M*M complex,
 * row-major) without allocating anything: its only scratch, one contraction
 * vector per node (the sum of all bond ranks, at most 65536 complex values), is
 * a fixed 1 MiB array compiled into the library, which every GPU that loads the
 * library keeps until the process exits. A tree needing more is refused with
 * TTN_EINVAL and a message in err (err_len bytes; err may be NULL).
 * node_dev[u] points to node u's tensor in canonical layout (the layout
 * ttn_get_node returns); tree, leg_dims and ranks are as for ttn_create. The
 * first call on each device looks up the array's device address with that
 * device current; make that first call before any CUDA stream capture. The
 * address is kept for the life of the process, so do not call this again on a
 * device after cudaDeviceReset. Devices beyond ordinal 63 get TTN_EINVAL. All
 * calls on one device share the array, which keeps the last call's contents;
 * every entry a call reads it has written first, so nothing needs clearing.
 * Calls that overlap on the GPU (different streams or host threads) race on
 * the array. Work is issued on `stream` (a cudaStream_t passed as void*); the
 * call does not synchronise. */
ttn_status ttn_rdm_noalloc(const ttn_tree* tree, const int32_t* leg_dims, const int32_t* ranks,
                           const void* const* node_dev, void* rho_dev, void* stream, char* err,
                           size_t err_len);

/* Autotuner (no counterpart in the paper: GB300 work distribution). Times
 * every CUDA-core contraction job list of the handle on its stream with each
 * admissible tile shape -- warps per CTA w in {8, 4, 2} sharing one 32-output
 * tile, times the split k = 1 .. min(useful(w), max_split) CTAs (one cluster)
 * per tile -- and keeps the fastest (another shape must win by 3 %); the
 * environment projections get the split only. Lists with the same key (see
 * ttn_tuning_get) are timed once and share the shape. reps timed launches per shape,
 * after one warm-up. The state is not modified: scratch-writing lists run as
 * they are, RK4 epilogue lists run as stage 1 into scratch, and the
 * environment matrices the projections overwrite are rebuilt before the next
 * step. Results stay within rounding of the untuned ones (reduction orders
 * change with the shape) and are deterministic for a given tuning. Changing
 * max_split or tile_warps, or a ps2 rank change rebuilding a list, returns
 * those lists to the planned shapes. reps: 1..100. Errors: TTN_ESTATE before
 * ttn_set_workspace, TTN_EINVAL. */
ttn_status ttn_autotune(ttn_t h, int32_t reps);

/* Tile shapes of the job lists, for caching a tuning across runs. Each list is
 * one row of TTN_TUNING_COLS int32: kind (0 contraction, 1 environment
 * projection), precision of the list (0 FP64, 1 FP32), the shape of its first
 * output (d0, d1, d2, d3; for projections d0, d1, d2 and the open leg), its
 * number of outputs, of terms (0 for projections) and of output tiles -- the
 * key of the row, 9 values -- then w (warps per CTA) and k (CTAs per tile).
 * ttn_tuning_get writes min(n_lists, max_rows) rows to rows (nullable when
 * max_rows is 0) and the number of lists to *n_rows. ttn_tuning_set gives
 * every list whose key equals a row's key that row's shape (the first such
 * row); *n_applied (nullable) = lists set. Rows with w not in {2, 4, 8} (8 for
 * projections) or k outside 1..max_split are refused with TTN_EINVAL before
 * anything is set. Errors: TTN_ESTATE before sop_load, TTN_EINVAL. */
#define TTN_TUNING_COLS 11

/* Tile shape of a batch (no counterpart in the paper): times reps batched ps1
 * steps of the handles (ttn_batch_step, after one untimed step that captures
 * the graphs) with tile_warps = 8, 4 and 2 on every member, keeps the fastest
 * (another must win by 3 %) and puts every member's state back (checkpoint
 * blobs in host memory) together with its ttn_stats counters, so the batch
 * continues from where it was. The members'
 * lists get the planned shapes for that warp count. *warps_out (nullable): the
 * warps chosen; ms_out (nullable, 3 floats): ms per batched step for 8, 4, 2.
 * Synchronises the members' streams. Errors: as ttn_batch_step, TTN_EINVAL for
 * reps outside 1..100. */
ttn_status ttn_batch_autotune(ttn_t* hs, int32_t n, double dt, int32_t reps, int32_t* warps_out, float* ms_out);
ttn_status ttn_tuning_get(ttn_t h, int32_t* rows, int32_t max_rows, int32_t* n_rows);
ttn_status ttn_tuning_set(ttn_t h, const int32_t* rows, int32_t n_rows, int32_t* n_applied);

/* Singular value decomposition a = U diag(sigma) V^H of a device matrix by
 * one-sided (Hestenes) Jacobi rotations in FP64: the factorisation the ps2
 * scheme uses to split a merged pair (Sec. 2.3, last paragraph), exposed for
 * callers and tests. a_dev: m x n complex, row-major (not modified); k =
 * min(m, n). Outputs: u_dev m x k and vh_dev k x n (device, row-major), sigma_host
 * k values in descending order; singular vectors of sigma = 0 are returned as
 * zero. ws_dev: ttn_svd_workspace_size(m, n) bytes, 256-byte aligned. Matrices
 * whose smaller side has more than 16 columns run over several CTAs (the pairs
 * of each round of the circle ordering spread over the CTAs, one barrier per
 * round: a thread-block cluster's up to 32 columns, else a cooperative launch
 * over the whole GPU); every grid barrier wait is bounded by wait_s seconds
 * (0..60). *sweeps_out (nullable): sweeps that rotated.
 * Synchronises `stream` (cudaStream_t as void*). Errors: TTN_EINVAL,
 * TTN_ENOMEM (workspace too small or misaligned), TTN_ETIMEOUT (a barrier
 * wait gave up; outputs undefined), TTN_ENUMERIC (no convergence within 60
 * sweeps), TTN_ECUDA. */
ttn_status ttn_svd_workspace_size(int32_t m, int32_t n, size_t* bytes);
ttn_status ttn_svd(const void* a_dev, int32_t m, int32_t n, void* u_dev, double* sigma_host, void* vh_dev,
                   void* ws_dev, size_t ws_bytes, double wait_s, int32_t* sweeps_out, void* stream);

const char* ttn_last_error(ttn_t h);
/* Waits for the work queued on the handle's stream (a step that failed part-way
 * may have left launches behind), then frees the handle's host resources,
 * graphs and events. The caller frees the workspace afterwards. */
void ttn_destroy(ttn_t h);

#ifdef __cplusplus
}
#endif
#endif /* TTN_HEOM_H */
