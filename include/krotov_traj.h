/*
 * krotov_traj.h — C ABI of the trajectory-parallel Krotov library for GB300 (sm_103a).
 *
 * Method: Goerz & Jacobs, "Efficient optimization of state preparation in quantum networks
 * using quantum trajectories" (arXiv:1801.04382).  The library runs, on one GPU, the
 * independent-trajectory formulation of Krotov's method (Sec. 2.3): M quantum-jump (MCWF)
 * trajectories are propagated forward under the non-Hermitian effective Hamiltonian
 * (Sec. 2.1), co-states are propagated backward under its adjoint, and the pulse is updated
 * sequentially in time from the cross-trajectory sum of Im<chi_k|dH/deps_i|psi_k>
 * (Eq. independent_traj_update), or, with kt_config.update_rule = 1, from the sum over all pairs
 * of trajectories of Eq. cross_traj_update.  Also: the exact gradient of the trajectory
 * functional (krotov_gradient), Krotov iterations as CUDA graph launches (krotov_update),
 * batches of independent problems (krotov_init_batch), the pulse noise measure of Eq. noise.
 *
 * General conventions
 *  - All pointers in the descriptors are HOST pointers; the library copies what it needs at
 *    krotov_init and never keeps a caller pointer.  Output pointers are host pointers written
 *    before the call returns (such calls synchronise the stream), except where a parameter is
 *    marked DEVICE (krotov_gradient, krotov_set_pulses_device, krotov_get_JT; krotov_set_uniforms
 *    takes either): those are read or written on `stream` without a host round trip.
 *  - Complex numbers are stored as two consecutive doubles (re, im).
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.  All
 *    device work of a call is enqueued on that stream.
 *  - The library owns every device buffer of a problem; krotov_free releases them.
 *  - Errors: every entry point returns a kt_status; no exception crosses the ABI.  A
 *    human-readable message for the calling thread's last error is returned by
 *    krotov_last_error().  Device-side failures (non-finite values, a full jump record, a
 *    pulse outside the spectral bound) are collected in a status word read at the end of
 *    each sweep and returned from that call.
 *  - One problem object must not be used from two threads at the same time.
 *
 * Limits: n_nodes <= 8, n_loc <= 16, n_ctrl <= 8, n_lind <= 4, n_pairs <= 28,
 * d = n_loc^n_nodes must fit two tile buffers in 227 KB of shared memory
 * (d <= ~14000 in FP32-mixed, ~7000 in FP64 for one trajectory per CTA).
 */
#ifndef KROTOV_TRAJ_H
#define KROTOV_TRAJ_H

#ifdef __cplusplus
extern "C" {
#endif

#define KT_API __attribute__((visibility("default")))

typedef struct kt_problem kt_problem;   /* opaque; created by krotov_init, owned by the library */
typedef struct kt_batch kt_batch;       /* opaque; independent problems iterated together */

typedef enum {
  KT_OK = 0,
  KT_ERR_ARG = -1,          /* invalid argument or descriptor */
  KT_ERR_OOM = -2,          /* device allocation failed */
  KT_ERR_CUDA = -3,         /* a CUDA runtime call failed */
  KT_ERR_TIMEOUT = -4,      /* a bounded device-side wait expired */
  KT_ERR_NONFINITE = -5,    /* a NaN/Inf appeared in a norm, overlap or pulse */
  KT_ERR_RECORD_FULL = -6,  /* a trajectory needed more jumps than draws_per_traj allows */
  KT_ERR_STATE = -7,        /* call out of order (e.g. an updating forward pass without a backward pass) */
  KT_ERR_RANGE = -8,        /* a pulse value left [-eps_bound, eps_bound] */
  KT_ERR_UNSUPPORTED = -9   /* sizes beyond the limits above */
} kt_status;

typedef enum { KT_FP64 = 0, KT_FP32_MIXED = 1 } kt_precision;

/*
 * Model: a network of n_nodes identical-dimension nodes (paper Sec. 3.1), full space of
 * dimension d = n_loc^n_nodes, node 0 the most significant tensor factor.  The Hermitian
 * Hamiltonian is
 *     H(eps) = sum_i h0_i + sum_c eps_c hc_c + sum_p coef_p a_{dst_p}^dag a_{src_p},
 * each h0_i / hc_c an n_loc x n_loc factor acting on one node (hc_c on node ctrl_node[c]),
 * `a` a single-node factor with at most one nonzero per row and per column (a ladder
 * operator, e.g. the cavity annihilation operator), and the pair list Hermitian as a whole
 * (Eq. ham_interaction is such a list).  Lindblad operators are L_l = sum_i lind_coef[l][i] a_i
 * (Sec. 3.1: one collective operator sqrt(2 kappa) sum_i a_i).  The library forms the MCWF
 * generator H_eff = H - (i/2) sum_l L_l^dag L_l (Sec. 2.1) in the same structured form.
 */
typedef struct {
  int n_nodes;
  int n_loc;
  const double *h0_local;   /* [n_nodes][n_loc][n_loc][2] drift factor of each node (Hermitian) */
  int n_ctrl;
  const int *ctrl_node;     /* [n_ctrl] node each control acts on */
  const double *hc_local;   /* [n_ctrl][n_loc][n_loc][2] control factor dH/deps_c (Hermitian) */
  const double *a_local;    /* [n_loc][n_loc][2] ladder factor used by pairs and Lindblad ops */
  int n_pairs;
  const int *pair_dst;      /* [n_pairs] */
  const int *pair_src;      /* [n_pairs], != pair_dst */
  const double *pair_coef;  /* [n_pairs][2] */
  int n_lind;
  const double *lind_coef;  /* [n_lind][n_nodes][2] */
  const double *psi0;       /* [d][2] initial state of every trajectory, or NULL if psi0_batch */
  const double *psi0_batch; /* [M][d][2] per-trajectory initial states, or NULL */
  const double *psi_tgt;    /* [d][2] target state (normalised by the caller) */
} kt_model_desc;

/*
 * Run configuration.  Time grid t_j = j T / nt, controls piecewise constant on the nt
 * intervals (Sec. 2.2).  Uniform random numbers (Sec. 2.1: r in [0,1) for the norm threshold
 * and the channel choice) are supplied by the caller: forward pass p uses row
 * uniforms[p mod n_passes][k][.] for trajectory k — column 0 is the first threshold r, and
 * after the m-th jump column 2m-1 chooses the channel and column 2m is the next r.  At most
 * (draws_per_traj - 1) / 2 jumps per trajectory and pass.
 */
typedef struct {
  double T;
  int nt;
  int M;                    /* number of trajectories */
  kt_precision prec;        /* KT_FP64, or KT_FP32_MIXED: complex64 states with FP32
                               arithmetic, FP64 norms, renormalisation, overlaps and sums */
  int ckpt_interval;        /* 0: keep the co-state at every t_j; K > 0: keep every K-th
                               and recompute the rest segment by segment; -1: automatic from the
                               device memory free at krotov_init -- every co-state if they fit,
                               else the longest prefix t_0..t_A plus checkpoints every K after it
                               with the fewest recomputed co-states (a reserve of max(2 GiB, 2 %)
                               and 2 sqrt(nt) + 4 states stays free); krotov_get_info reports the
                               choice.  Results are bit-identical whatever the storage. */
  const double *eps_guess;  /* [n_ctrl][nt] guess pulse eps_c^(0) on each interval */
  const double *shape;      /* [n_ctrl][nt] update shape S_c(t_{j-1/2}) in [0, 1] */
  const double *lambda_a;   /* [n_ctrl] Krotov step weights lambda_c > 0 */
  const double *uniforms;   /* [n_passes][M][draws_per_traj] values in [0, 1) */
  int n_passes;
  int draws_per_traj;       /* odd, >= 1 */
  double eps_bound;         /* bound on |eps| used for the spectral estimate; 0 = automatic
                               (2 max|eps_guess| + 1) */
  double cheb_tol;          /* Chebyshev truncation; 0 = 1e-16 (FP64) / 2^-24 (FP32-mixed) */
  int tile_traj;            /* trajectories per CTA tile (power of two <= 32); 0 = automatic
                               (heuristic); -1 = autotuned: krotov_init times the forward
                               interval kernel for every width that fits (12 launches each on
                               `stream`, guess pulse) and keeps the fastest */
  int update_rule;          /* 0: independent-trajectory update (Eq. independent_traj_update),
                               co-states chi_k(T) = tau_k |tgt>; 1: cross-trajectory update
                               (Eq. cross_traj_update), co-states xi_k(T) = |tgt> and
                               Delta eps_c = S_c / (M^2 lambda_c) sum_{k,k'}
                               Im[<xi_k|h_c|psi_k'><psi_k'|xi_k>] (all pairs of trajectories) */
  int jump_scheme;          /* 0: jump times located by bisection of the norm, several jumps per
                               interval possible (Sec. 2.1); 1: the first-order scheme of Sec. 2.1,
                               at most one jump per interval, applied at its end (s* = dt) */
  int ckpt_prefix;          /* with ckpt_interval = K > 0: the co-states of t_0 .. t_ckpt_prefix
                               are all kept as well (checkpoints every K after it); 0 = none */
  int traj_offset;          /* trajectory sharding (Sec. 2.3: trajectories are independent, only the
                               update's scalars are exchanged): with M_total > 0 this problem is the
                               shard holding trajectories traj_offset .. traj_offset + M - 1 of an
                               M_total-trajectory problem -- its uniforms are those trajectories' rows,
                               Delta eps is normalised by M_total, and the per-interval tile partials
                               of all shards are exchanged (krotov_shard_nccl, or a group of shards in
                               one process, krotov_group_init) before Delta eps is formed, in the same
                               order as the unsharded problem (bit-identical results).  Shard
                               boundaries fall on tile boundaries; the tile width is chosen for
                               M_total (tile_traj -1 is refused); independent update rule only. */
  int M_total;              /* 0: not a shard */
  int inject_copy_timeout;  /* 0 (normal).  1: a test of failure reporting -- every interval kernel's
                               first bounded wait for a state tile's bulk copy watches a barrier that
                               nothing arrives at (about 10 us), takes its timeout path (a second wait
                               lets the copy land, the block leaves) and the sweep returns
                               KT_ERR_TIMEOUT; the device stays usable.  Each wait is bounded
                               (about 2 s) whatever this flag. */
  int items_per_thread;     /* thread mapping of the interval kernels.  0 = automatic: for the node
                               dimensions 6 and 9 one thread per last-node fiber (the cavity-structure
                               kernels when the generator has that structure) -- unless a trajectory has
                               fewer than 16 fibers and the tile width is automatic too, then the strided
                               mapping with one item per thread -- else the strided mapping with the
                               fewest items per thread that fit; with tile_traj = -1 the autotuner also
                               times the strided mapping at 1, 2 and 4 items per thread.
                               1, 2, 4, 8 or 16: the strided mapping (item q of thread t is element
                               t + q * threads of the tile) with that many items per thread -- more
                               threads per trajectory for problems too small to fill the GPU otherwise */
  int per_interval_launches; /* 0 = automatic: when the problem runs on the strided mapping, every tile
                               is resident on the GPU at once and every co-state is kept (small
                               problems), each sweep is one
                               launch -- the backward sweep a plain one, the forward sweep a cooperative
                               one whose CTAs meet at a grid barrier after each interval to form the
                               update (Sec. 2.2: the update of interval j+1 needs every trajectory's
                               state at t_j); bit-identical to the per-interval launches.  Not used for
                               shards, the cross-trajectory rule, the sweeps that keep states for the
                               gradient, or the problems of a batch.  1 = one launch per interval. */
} kt_config;

/* Create a problem: validate, assemble H_eff in structured form (a1), choose the Chebyshev
 * expansion (a2), allocate and upload.  No propagation is done. */
KT_API kt_status krotov_init(const kt_model_desc *model, const kt_config *cfg, void *stream,
                             kt_problem **out);

/* Density-matrix Krotov (Sec. 2.2, Eqs. krotov_functional, krotovupdate, krotov_boundary), the
 * convergence reference of the trajectory methods: rho(t) follows the master equation of Eq. lindblad,
 * d rho/dt = -i (H_eff rho - rho H_eff^dag) + sum_l L_l rho L_l^dag, with the model's H, L_l (the same
 * descriptor as krotov_init, pure initial state psi0); the functional is J_T = 1 - <tgt|rho(T)|tgt>,
 * the co-state P(t) runs backward from P(T) = |tgt><tgt| under the adjoint dynamics, and the
 * sequential update is Delta eps_c(t) = S_c / lambda_c Im <<P(t)| [H_c, rho(t)] >> with
 * <<A|B>> = tr(A^dag B) and dL/deps_c rho = [H_c, rho] as the paper states it.
 * The library runs it as ONE state vec(rho)[x d + y] = rho_xy of a network of 2 n_nodes nodes (ket
 * nodes, then bra nodes) under G = H_eff (x) 1 - 1 (x) H_eff^* + i sum_l L_l (x) L_l^*
 * (d vec(rho)/dt = -i G vec(rho)), with the trajectory kernels: no jumps, no normalisation.  So
 * propagate_forward / propagate_backward / krotov_update / krotov_get_update / krotov_get_pulses
 * work as for a trajectory problem; fidelity's F is <tgt|rho(T)|tgt> (tau_out[0] = <<P_tgt|rho(T)>>),
 * krotov_get_states returns vec(rho(T)) as [1][d*d][2] and krotov_get_costate vec(P(t_j)).
 * cfg: T, nt, prec, ckpt_interval (and ckpt_prefix), eps_guess, shape, lambda_a, eps_bound and
 * cheb_tol are used; M, the uniforms, tile_traj, update_rule and jump_scheme are ignored.
 * Limits: n_nodes <= 4, d^2 within the shared-memory limit above (two states of d^2 elements:
 * d <= 81 in FP64), a real ladder factor.  krotov_gradient and the cross-trajectory rule are not
 * defined for it (KT_ERR_UNSUPPORTED / KT_ERR_ARG). */
KT_API kt_status krotov_init_density(const kt_model_desc *model, const kt_config *cfg, void *stream,
                                     kt_problem **out);

/* One forward MCWF sweep of all trajectories over [0, T] (Sec. 2.1), consuming the next
 * pass of uniforms.  sequential_update = 0 propagates under the current pulse.
 * sequential_update = 1 applies Krotov's update (Eq. independent_traj_update) on the fly:
 * before interval j is propagated, Delta eps_cj = S_cj / (lambda_c M) sum_k
 * Im <chi_k(t_{j-1})| hc_c |psi_k(t_{j-1})> is formed from the co-states of the preceding
 * propagate_backward, and the new pulse eps + Delta eps drives interval j; it becomes the
 * current pulse when the sweep ends.  Requires a backward sweep since the last forward sweep.
 * At the end tau_k = <tgt|psi_k(T)>/||psi_k(T)|| is formed; F_out (nullable) receives
 * F = (1/M) sum |tau_k|^2 (Eq. functional_traj). */
KT_API kt_status propagate_forward(kt_problem *p, int sequential_update, double *F_out, void *stream);
/* sequential_update = 2: a sweep without update that also keeps the forward states (every
 * ckpt_interval intervals, or all of them when ckpt_interval = 0) for krotov_gradient.  Any
 * later forward sweep or krotov_set_pulses discards them. */

/* Exact gradient dJ_T/deps_ij (Sec. 2.2, Eq. gradient: the discrete derivative of the propagator)
 * of the trajectory functional J_T = 1 - (1/M) sum_k |<tgt|psi_k(T)>|^2 / ||psi_k(T)||^2
 * (Eq. functional_traj), for the jump record of a forward sweep held fixed:
 *   dJ_T/deps_ij = -(2/M) sum_k Re <chi~_k(t_j)| dU_kj/deps_i |psi_k(t_{j-1})>,
 * chi~_k(T) = (tau_k |tgt> - |tau_k|^2 psihat_k) / ||psi_k(T)||, chi~ propagated backwards along
 * each trajectory's own record, dU/deps exact.  Forward states are replayed segment by segment from
 * the kept ones.
 *   eps_dev  DEVICE [n_ctrl][nt] pulse, or NULL.  Non-NULL: the pulse is set from it (as
 *            krotov_set_pulses_device) and a forward sweep that keeps its states runs first (it
 *            consumes the next pass of uniforms); the gradient is that sweep's.  NULL: the gradient
 *            of the last propagate_forward(p, 2, ...) at the current pulse (KT_ERR_STATE if none).
 *   dJ_dev   DEVICE [n_ctrl][nt] output, written on `stream` (the caller owns it).
 * Everything stays on the device; the call synchronises `stream` once to read the status word.
 * Needs four state buffers of d in shared memory (KT_ERR_UNSUPPORTED otherwise). */
KT_API kt_status krotov_gradient(kt_problem *p, const double *eps_dev, double *dJ_dev, void *stream);

/* Replace the current pulse from DEVICE memory eps_dev [n_ctrl][nt] (device-to-device copies on
 * `stream`, no host round trip); invalidates co-states, records and kept states like
 * krotov_set_pulses.  The values are checked on the device (finite, |eps| <= eps_bound); a failure
 * is reported by the next sweep as KT_ERR_NONFINITE / KT_ERR_RANGE. */
KT_API kt_status krotov_set_pulses_device(kt_problem *p, const double *eps_dev, void *stream);

/* J_T = 1 - (1/M) sum_k |tau_k|^2 of the last forward sweep (Eq. functional_traj) written to one
 * DEVICE double JT_dev on `stream` (no synchronisation). */
KT_API kt_status krotov_get_JT(kt_problem *p, double *JT_dev, void *stream);

/* Backward co-state sweep (Sec. 2.3): chi_k(T) = tau_k |tgt>, then
 * chi_k(t_{j-1}) = U_kj^dag chi_k(t_j) under the pulse of the last forward sweep, where U_kj
 * is trajectory k's own forward map over interval j including its recorded jumps c L_l.
 * Requires a forward sweep. */
KT_API kt_status propagate_backward(kt_problem *p, void *stream);

/* n_iter Krotov iterations, each = propagate_backward + propagate_forward(update = 1).  If
 * no forward sweep has run yet, a guess sweep propagate_forward(0) runs first.  JT_out and
 * J_out (nullable, [n_iter]) receive J_T = 1 - F and Krotov's functional
 * J = J_T + sum_c lambda_c sum_j Delta eps_cj^2 dt / S_cj (Eq. krotov_functional, S = 0
 * points skipped) after each iteration.  With profiling off, each iteration is one CUDA graph
 * launch: the launches of an iteration are captured on first use for each state of the
 * double-buffered pulse and record arrays (two alternate), and device failures are reported at
 * the end of the iteration instead of after each sweep.  The results are identical to calling
 * propagate_backward and propagate_forward(p, 1, ...) in turn. */
KT_API kt_status krotov_update(kt_problem *p, int n_iter, double *JT_out, double *J_out, void *stream);

/* F and tau_k ([M][2], nullable) of the last forward sweep (Eq. functional_traj). */
KT_API kt_status fidelity(kt_problem *p, double *F_out, double *tau_out);

/* Current pulse [n_ctrl][nt], and the update Delta eps [n_ctrl][nt] of the last updating
 * forward sweep (zeros before the first). */
KT_API kt_status krotov_get_pulses(kt_problem *p, double *eps_out);
KT_API kt_status krotov_get_update(kt_problem *p, double *deps_out);
/* Replace the current pulse (host array [n_ctrl][nt]); invalidates co-states and records. */
KT_API kt_status krotov_set_pulses(kt_problem *p, const double *eps);

/* Jump record of the last forward sweep.  count_out [M]; step_out/channel_out/s_out/c_out
 * [M][max_jumps] (any may be NULL): 1-based interval index j, Lindblad channel l, offset s*
 * of the jump from t_{j-1}, and the renormalisation c = 1/||L_l psi(s*)||. */
KT_API kt_status krotov_get_records(kt_problem *p, int *count_out, int *step_out, int *channel_out,
                                    double *s_out, double *c_out);

/* Final states psi_k(T) of the last forward sweep, [M][d][2] (not normalised). */
KT_API kt_status krotov_get_states(kt_problem *p, double *psi_out);
/* Co-state chi_k(t_j), [M][d][2], of the last backward sweep; only for ckpt_interval = 0 or
 * j a checkpoint. */
KT_API kt_status krotov_get_costate(kt_problem *p, int j, double *chi_out);

/* Noise of the current pulse (Eq. noise): nu_out[c] = sum_j |e_cj - smooth_cj| dt for each control
 * (host output [n_ctrl]), e = eps, or eps - ref when ref (host [n_ctrl][nt], nullable) is given --
 * e.g. ref = the guess pulse measures the noise of the accumulated update without the smoothing
 * residual of a smooth guess.  smooth = five-point cubic Savitzky-Golay smoothing (the
 * least-squares cubic through the five samples centred on j, or the first / last five at the two
 * ends, evaluated at j).  Computed on the device from the device-resident pulse; needs nt >= 5
 * (KT_ERR_ARG otherwise).  Synchronises `stream`. */
KT_API kt_status krotov_pulse_noise(kt_problem *p, const double *ref, double *nu_out, void *stream);

/* Replace the uniform random numbers ([n_passes][M][draws_per_traj] in host OR device memory --
 * the copy direction is taken from the pointer; 1 <= n_passes <= the value given at init, draws as
 * at init); later passes cycle through these n_passes rows, starting again at row 0.  Asynchronous
 * on `stream`; the array must stay valid until the stream reaches the copy (pinned host memory or
 * device memory). */
KT_API kt_status krotov_set_uniforms(kt_problem *p, const double *uniforms, int n_passes, void *stream);

/* Per-launch timing of the interval kernels with CUDA events recorded on the calling stream
 * around every launch (on = 1), e.g. to derive each kernel's average duration during a
 * benchmark.  Turning it on or off clears the totals.  krotov_get_profile returns, per family
 * (KT_PROF_FWD: forward interval kernel incl. the pulse update; KT_PROF_BWD: backward interval
 * kernel incl. checkpoint recompute and the gradient's forward replay; KT_PROF_GRAD: gradient
 * kernel of krotov_gradient; KT_PROF_CROSS: the cross-trajectory update's kernels; KT_PROF_FINISH:
 * the one-block update sum of a sharded problem), the summed
 * milliseconds and
 * the launch count since profiling was turned on; arrays of KT_PROF_FAMILIES entries. */
#define KT_PROF_FWD 0
#define KT_PROF_BWD 1
#define KT_PROF_GRAD 2
#define KT_PROF_CROSS 3
#define KT_PROF_FINISH 4
#define KT_PROF_FAMILIES 5
KT_API kt_status krotov_set_profiling(kt_problem *p, int on);
KT_API kt_status krotov_get_profile(kt_problem *p, double *ms_out, long long *launches_out);

/* Sizes chosen at init: max jumps per pass, Chebyshev terms per step, tile width, tiles,
 * threads per CTA, and the spectral interval [e_min, e_max] of the forward generator's
 * Hermitian part; passes = completed forward sweeps since the uniforms were last uploaded (pass
 * p used row p mod n_passes), which lets a run be resumed bit-identically: a new problem with the
 * saved pulse, the same eps_bound and the uniform rows from passes - 1 on repeats the last forward
 * sweep exactly. */
typedef struct {
  int d, max_jumps, cheb_terms, tile_traj, n_tiles, threads;
  double e_min, e_max, damping;
  long long device_bytes;
  long long passes;
  double eps_bound;         /* the pulse bound the spectral estimate used (given or automatic) */
  long long sweeps;         /* forward sweeps completed since krotov_init (never reset): tells a
                               caller whether another sweep ran since the one it depends on */
  int ckpt_interval;        /* co-state storage in use: 0 = every co-state kept; K > 0 = the
                               co-states of t_0 .. t_{ckpt_kept_prefix} kept, then every K-th */
  int ckpt_kept_prefix;
  int costate_slots;        /* co-state slots held in device memory */
  int items_per_thread;     /* thread mapping of the interval kernels: 0 = one thread per last-node
                               fiber, else the strided mapping with this many items per thread */
  int whole_sweep;          /* 1: sweeps run as one launch each (see kt_config.per_interval_launches) */
} kt_info;
KT_API kt_status krotov_get_info(kt_problem *p, kt_info *info);

KT_API void krotov_free(kt_problem *p);
KT_API const char *krotov_last_error(void);

/* Batches of independent optimisation problems (the trajectories of one problem are
 * independent of every other problem, Sec. 2.3), e.g. networks of different sizes.
 * krotov_init_batch creates n problems as krotov_init would (models[i] with cfgs[i]; on failure
 * nothing is kept and the message names the problem index).  krotov_batch_update runs n_iter
 * Krotov iterations of every problem; each iteration is ONE CUDA graph launch on `stream` whose
 * branches are the problems' captured iterations, with no dependency between problems, so that
 * the device runs the problems' interval kernels concurrently.  Problems without a forward
 * sweep first run their guess sweeps, concurrently on internal streams.  JT_out (nullable,
 * [n_iter][n]) receives 1 - F of each problem after each iteration.  Results are identical to
 * krotov_update on each problem alone.  krotov_batch_problem lends problem i (owned by the
 * batch: use it with the single-problem calls, never free it); krotov_batch_info reports the
 * problem count, the kernel nodes of the last built batch graph and the device bytes held. */
KT_API kt_status krotov_init_batch(const kt_model_desc *const *models, const kt_config *const *cfgs, int n,
                                   void *stream, kt_batch **out);
KT_API kt_status krotov_batch_update(kt_batch *b, int n_iter, double *JT_out, void *stream);
KT_API kt_status krotov_batch_problem(kt_batch *b, int i, kt_problem **out);
KT_API kt_status krotov_batch_info(kt_batch *b, int *n_problems, long long *graph_nodes,
                                   long long *device_bytes);
KT_API void krotov_batch_free(kt_batch *b);

/* Trajectory sharding across GPUs (Sec. 2.3: the trajectories are independent and only scalars are
 * exchanged).  Each process creates its shard with kt_config.traj_offset / M_total (equal slices in
 * rank order: M_total = world * M, traj_offset = rank * M), then joins the communicator:
 *   kt_nccl_unique_id   on one rank: a 128-byte NCCL unique id into id_out (host), to be sent to the
 *                       other ranks by the caller's own means;
 *   krotov_shard_nccl   on every rank, with its device current: a communicator of `world` ranks.
 * From then on every updating forward sweep all-gathers the tile partials of the update overlap once
 * per interval (in place, n_tiles x n_ctrl doubles per shard) and every shard forms the same Delta eps;
 * each forward sweep ends with an all-gather of tau, so F (fidelity, krotov_update's J_T) is that of
 * all M_total trajectories.  The collectives are enqueued on the sweep's stream and captured into
 * krotov_update's graphs.  NCCL is loaded at run time (nccl_library, or "libnccl.so.2" when NULL);
 * KT_ERR_UNSUPPORTED if it cannot be loaded.  The communicator is destroyed by krotov_free. */
KT_API kt_status kt_nccl_unique_id(const char *nccl_library, void *id_out);
KT_API kt_status krotov_shard_nccl(kt_problem *p, const void *unique_id, int rank, int world,
                                   const char *nccl_library);

/* Shards of one problem driven together in one process, on one stream (e.g. one device): the group
 * runs their forward sweeps interval by interval, copies each shard's tile partials into every other
 * shard's copy of the global partials (device-to-device) and forms Delta eps in every shard; the
 * backward sweeps are independent.  krotov_group_init borrows n shards (any order; together they
 * must cover trajectories 0 .. M_total - 1 in consecutive ranges with one tile width);
 * krotov_group_update runs n_iter Krotov iterations (a guess sweep first if needed), JT_out
 * (nullable, [n_iter]) gets J_T of all trajectories after each; krotov_group_fidelity gives F of the
 * last sweep over all trajectories.  Each shard's own getters (pulses, records, states) work as usual;
 * its propagate_* / krotov_update calls are refused while it has no communicator.  krotov_group_free
 * releases the group, not the shards.  The results equal the unsharded problem's bit for bit. */
typedef struct kt_group kt_group;
KT_API kt_status krotov_group_init(kt_problem *const *shards, int n, kt_group **out);
KT_API kt_status krotov_group_update(kt_group *g, int n_iter, double *JT_out, void *stream);
KT_API kt_status krotov_group_fidelity(kt_group *g, double *F_out, void *stream);
KT_API void krotov_group_free(kt_group *g);

/* Chebyshev coefficient helper (host): Bessel J_0..J_{n-1}(alpha) by Miller's backward
 * recurrence, the routine the kernels use for sub-step propagators.  Returns KT_ERR_ARG for
 * alpha < 0 or n outside [1, 256]. */
KT_API kt_status kt_bessel_j(double alpha, int n, double *out);

/* Host-only check helper: the structured generator tables built by krotov_init for the given
 * model and configuration, expanded into a dense matrix out [d][d][2] with the same indexing the
 * kernels use (every neighbour index bounds-checked; KT_ERR_RANGE if one leaves the space).
 * direction 0: H_eff(eps) = H(eps) - (i/2) sum_l L_l^dag L_l (Sec. 2.1); direction 1: -H_eff(eps)^dag,
 * the generator of the backward co-state propagation; directions 2 and 3: the same for the
 * Liouville-space generator G of krotov_init_density (out is then [d^2][d^2][2]).  eps: [n_ctrl]
 * pulse values.  No device call. */
KT_API kt_status kt_generator_dense(const kt_model_desc *model, const kt_config *cfg, int direction,
                                    const double *eps, double *out);

/* Allocation-free pulse-update reduction (the paper has no counterpart: this is a library
 * service).  For callers that may not allocate device memory -- e.g. a host framework that owns
 * and budgets every device allocation up front, or code running from a callback where
 * cudaMalloc is not allowed -- this computes the same per-interval update as the forward
 * sweep, Delta eps_c = shape_j[c] / (lambda_a[c] M) sum_k Im <chi_k| hc_c |psi_k>, without
 * allocating anything: its scratch (1024 block partials x 8 controls + a ticket, 64 KB) is a
 * fixed device array inside the library, held by every GPU that loads the library until the
 * process exits.
 *   psi, chi   DEVICE pointers, [M][d][2] FP64 states (plain layout, d = n_loc^n_nodes)
 *   hc_local   HOST [n_ctrl][n_loc][n_loc][2] control factors, ctrl_node [n_ctrl] (host)
 *   shape_j, lambda_a  HOST [n_ctrl];  deps_out DEVICE [n_ctrl] FP64 (written on `stream`)
 * Every call looks up the scratch array's device address on the current device (a host-only
 * query); the first call on a device may load the library's device code there, so make that
 * first call before any stream capture begins.  Every call shares the one array and
 * the call clears its ticket itself, so calls whose kernels overlap on the GPU (different
 * streams, or different host threads on the same device) race and must be serialised by the
 * caller.  Sizes beyond the scratch (n_ctrl > 8) are rejected with KT_ERR_UNSUPPORTED;
 * n_nodes <= 8, n_loc <= 16, d <= 2^24, at most 6 entries per control-factor row. */
KT_API kt_status kt_update_overlap_noalloc(int n_nodes, int n_loc, int n_ctrl, const int *ctrl_node,
                                           const double *hc_local, int M, const double *psi,
                                           const double *chi, const double *shape_j,
                                           const double *lambda_a, double *deps_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* KROTOV_TRAJ_H */
