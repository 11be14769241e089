/*
 * dpde.h -- C ABI of the GB300 DPDE timestep library (libdpde.so).
 *
 * Method: Dissipative Particle Dynamics with Energy conservation (DPDE) as
 * defined by Homman, Maillet, Roussel and Stoltz, "New parallelizable schemes
 * for integrating the Dissipative Particle Dynamics with Energy Conservation"
 * (arXiv:1507.06643). Section II.A, Eq. (DPDE), gives the dynamics of a
 * particle's position q_i, momentum p_i and internal energy eps_i; friction and
 * noise act on the full relative velocity (not projected on the line of
 * centres). Section III splits one timestep into a velocity-Verlet step of the
 * Hamiltonian part (Eq. newton) followed by a fluctuation/dissipation (FD) step
 * (Eq. DPDE_dissipative) integrated by one of the schemes of Sec. III.A/III.B.
 *
 * Everything below is plain C: pointers, sizes and status codes. The library
 * owns every device buffer it allocates; caller arrays are only read or
 * written during the call that receives them.
 *
 * ---------------------------------------------------------------------------
 * Units, model and conventions (reduced units, k_B = 1, dimension d = 3)
 * ---------------------------------------------------------------------------
 *  - Cut-off function, Eq. (pot_mou): chi(r) = (1 - r/r_cut)^2 for r < r_cut,
 *    else 0; the noise amplitude uses sqrt(chi) = 1 - r/r_cut. A pair
 *    interacts iff r^2 < r_cut^2 (chi, its root and the force all vanish at
 *    r_cut, so the strict inequality only matters to rounding).
 *  - Conservative potential: soft repulsion v(r) = (a r_cut / 2)(1 - r/r_cut)^2
 *    for r < r_cut, force on i from j: a (1 - r/r_cut) (q_i - q_j)/r; a pair at
 *    r = 0 exerts no force. U = sum over pairs i<j of v(r_ij) (Eq.
 *    def_potential_energy with this v).
 *  - Equation of state, Eq. (DPDE_internalEOS) with constant heat capacity:
 *    eps_i = C_v T_i, so beta_i = 1/T_i = C_v / eps_i.
 *  - Fluctuation/dissipation relation, Eq. (DPDE_fd):
 *    gamma_ij = (sigma^2 / 4) (beta_i + beta_j).
 *  - Total energy (Sec. II.A): E = U + sum_i |p_i|^2 / (2 m) + sum_i eps_i.
 *    The paper prints the kinetic term without the 1/2; the kinetic energy
 *    variations of Eqs. (SSA_ij) and (SER_eint_discretization) fix it as
 *    |p|^2/(2m), which is what is conserved here.
 *  - Periodic boxes [0, L_x) x [0, L_y) x [0, L_z), minimum-image distances.
 *
 * ---------------------------------------------------------------------------
 * Particle identity and noise (Sec. III.A, the remark under Eq. SEM_fd; Sec.
 * III.B.1, the closing paragraph on regenerating G_ij^n)
 * ---------------------------------------------------------------------------
 *  - Particles of replica r are identified by id = 0 .. n_r-1, their index in
 *    the arrays handed to dpde_set_state (within that replica's segment).
 *  - The Gaussian increment of pair (i, j) at step n is a pure function of
 *    (seed, n, replica, min id, max id):
 *       x[0..3] = Philox4x32-10(counter = {id_min, id_max, (uint32)n, replica},
 *                               key     = {seed & 0xffffffff, seed >> 32})
 *    (Salmon, Moraes, Dror, Shaw, SC'11: multipliers 0xD2511F53, 0xCD9E8D57,
 *    Weyl key increments 0x9E3779B9, 0xBB67AE85, ten rounds).
 *    Uniforms with 24 significant bits, exact in float and double:
 *       u1 = ((x[0] >> 8) + 1) * 2^-24   in (0, 1]
 *       t1 = ( x[1] >> 8)      * 2^-24   in [0, 1)
 *       u2 = ((x[2] >> 8) + 1) * 2^-24,  t2 = (x[3] >> 8) * 2^-24
 *    Box-Muller: R_k = sqrt(-2 ln u_k);
 *       G = ( R1 cos(2 pi t1), R1 sin(2 pi t1), R2 cos(2 pi t2) ).
 *    G is G_ij for the ordered pair (id_min, id_max); G_ji = -G_ij. Tails are
 *    capped at |G_k| <= sqrt(48 ln 2) ~ 5.77.
 *
 * ---------------------------------------------------------------------------
 * One timestep (dpde_step), from state (q^n, p^n, eps^n) and F^n = F(q^n)
 * ---------------------------------------------------------------------------
 *  1. Velocity-Verlet (Sec. III.A, "standard Velocity-Verlet"):
 *       p <- p + (dt/2) F^n ;  q <- wrap(q + dt p / m)
 *       F^{n+1} = F(q^{n+1}) ;  p <- p + (dt/2) F^{n+1}
 *     wrap: x >= L -> x - L ; x < 0 -> x + L (one correction per step).
 *  2. Fluctuation/dissipation on the post-Verlet state with noise G^n
 *     (Trotter splitting, Appendix B.1: Hamiltonian part first):
 *       DPDE_SER    Eq. (SER_p) then Eq. (SER_eint_discretization): both sweeps
 *                   use the same pre-FD p and eps; updates are applied after
 *                   the second sweep. The energy update uses the factor -1/2
 *                   of Eq. (SER_eint_discretization) (Eq. SER_fd drops it; only
 *                   the -1/2 form conserves energy exactly).
 *       DPDE_HYBRID Sec. III.B.2: the SSA pair map of Eq. (SSA_ij) applied in
 *                   sequence to every interacting pair whose two particles lie
 *                   in the same domain ("processor"), in the order defined
 *                   below, then SER over all remaining (cross-domain) pairs on
 *                   the post-SSA state.
 *       DPDE_SEM    Eq. (SEM_fd) (Euler-Maruyama; does not conserve energy).
 *       DPDE_SSA    Eq. (SSA_ij) over all interacting pairs (Hybrid with one
 *                   domain spanning the periodic replica).
 *     The SSA map uses a = +2 gamma_ij chi dt / m (the printed minus sign is a
 *     typo: the map is the exact Ornstein-Uhlenbeck transition of
 *     p_ij = p_i - p_j at fixed gamma_ij, whose decay rate is 2 gamma chi / m);
 *     gamma_ij is evaluated from the current eps_i, eps_j of the sequence.
 *  3. n <- n + 1.
 *
 * ---------------------------------------------------------------------------
 * Cell grid, domains ("bricks") and the SSA order
 * ---------------------------------------------------------------------------
 *  For a replica with box L and brick grid B = (B_x, B_y, B_z):
 *       k_d     = floor(L_d / (B_d r_cut))   cells per brick along d (>= 1)
 *       ncell_d = B_d k_d                     (must be >= 3 and <= 1024)
 *       c_d(x)  = min(ncell_d - 1, (int)(x * (ncell_d / L_d)))
 *       brick_d = c_d / k_d
 *  The quotient ncell_d / L_d is formed once in double. A pair is "intra
 *  domain" (set A of Sec. III.B.2) iff both particles have the same brick.
 *  Order of the SSA sequence over A (the paper leaves it free, Sec. III.A.2):
 *   the cells are coloured per axis by their local coordinate l in the brick
 *   with period P_x = P_y = 3, P_z = 2 (the pairs of a cell reach offsets
 *   -1..1 along x and y but only 0..1 along z):
 *     col_d(l) = l mod P_d, except that along an axis where the brick spans
 *     the replica (B_d = 1, periodic) the last k_d mod P_d cells take colours
 *     P_d, P_d + 1;
 *   colours (col_z, col_y, col_x) are taken in lexicographic order (z major).
 *   The cells reached by the pairs of two cells of one colour are disjoint,
 *   so those cells are processed in any order. Within a cell, its particles i in
 *   ascending id, each applying its forward pairs (i, j) in the order
 *   (segment, id_j): j lies in a neighbour cell of the same brick (wrapping
 *   only along B_d = 1 axes) at offset (dx, dy, dz) with segment
 *   9 (dz+1) + 3 (dy+1) + (dx+1) above 13, or in i's own cell (segment 13)
 *   with id_j > id_i. DPDE_SSA uses the same order with the whole replica as
 *   one brick (B = (1, 1, 1), k = ncell).
 *
 * ---------------------------------------------------------------------------
 * Precision modes
 * ---------------------------------------------------------------------------
 *  DPDE_FP64  : every quantity in double.
 *  DPDE_MIXED : q, p, forces and pair arithmetic in float; eps in double. The
 *               internal-energy updates account in double for the kinetic
 *               energy change of the stored float momenta, so the FD part
 *               conserves the double-evaluated total energy to rounding of
 *               the per-particle antisymmetric pair sums (equal in exact
 *               arithmetic to Eq. SER_eint_discretization and Eq. SSA_ij).
 */
#ifndef DPDE_H
#define DPDE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes (every entry point returns one) ---- */
#define DPDE_OK                 0
#define DPDE_ERR_ARG           -1  /* invalid argument; nothing was changed   */
#define DPDE_ERR_CUDA          -2  /* CUDA runtime error (message kept)       */
#define DPDE_ERR_OOM           -3  /* device allocation failed                */
#define DPDE_ERR_NEG_EPS       -4  /* some eps_i <= 0 after the last step(s);
                                      the state was advanced, nothing clamped */
#define DPDE_ERR_NONFINITE     -5  /* NaN/Inf in the state                    */
#define DPDE_ERR_TIMEOUT       -6  /* a bounded device wait gave up: a grid
                                      barrier of the persistent SSA launch
                                      (ssa_mode 3) waited past the handle's
                                      wait budget; the step is incomplete     */
#define DPDE_ERR_CAPACITY      -7  /* a particle had more neighbours than the
                                      list holds (density far above the one
                                      the handle was sized for); the step's
                                      FD part is invalid                      */

/* ---- enumerations ---- */
#define DPDE_FP64   0
#define DPDE_MIXED  1

#define DPDE_SER     0
#define DPDE_HYBRID  1
#define DPDE_SEM     2
#define DPDE_SSA     3

/* Global model parameters (shared by all replicas of a handle). */
/* Pair potentials. DPDE_POT_SOFT: v = (a r_cut / 2)(1 - r/r_cut)^2.
 * DPDE_POT_LJ: the shifted, splined and truncated Lennard-Jones potential of
 * Eq. (Ep), v = 4 eps_LJ((r_LJ/r)^12 - (r_LJ/r)^6) - eps_sh - f_sp (r - r_cut)
 * below r_cut with eps_sh, f_sp fixed by v(r_cut) = v'(r_cut) = 0; r_cut is
 * the same cutoff as chi's (the paper writes both with r_cut). Coincident
 * particles (r = 0) exert no force; their LJ energy term is left out. */
#define DPDE_POT_SOFT 0
#define DPDE_POT_LJ   1

typedef struct dpde_params {
    double   mass;       /* m  > 0                                          */
    double   r_cut;      /* r_cut > 0: range of chi and of the potential    */
    double   a;          /* soft-repulsion amplitude a >= 0                 */
    double   sigma;      /* fluctuation strength sigma >= 0, Eq. (DPDE_fd)  */
    uint64_t seed;       /* Philox key                                      */
    int32_t  precision;  /* DPDE_FP64 or DPDE_MIXED                         */
    int32_t  potential;  /* DPDE_POT_SOFT (0) or DPDE_POT_LJ                */
    double   lj_eps;     /* eps_LJ >= 0 (DPDE_POT_LJ)                       */
    double   lj_r;       /* r_LJ > 0 (DPDE_POT_LJ)                          */
} dpde_params;

/* One independent system ("replica", one of the N_traj trajectories of
 * Eq. obs_time_estimation_traj). */
typedef struct dpde_replica {
    int64_t n;           /* number of particles, >= 0                       */
    double  box[3];      /* L_x, L_y, L_z > 0                               */
    double  cv;          /* constant heat capacity C_v > 0                  */
    int32_t bricks[3];   /* Hybrid domain grid B_d >= 1 (1,1,1 = one domain) */
    int32_t walls;       /* 0: periodic along z; 1: specular walls along z   */
    double  wall_u;      /* walls = 1: velocity of the upper wall (<= 0)     */
} dpde_replica;

/* Walls (the confining walls of the shock set-up, Sec. V, read as hard
 * specular walls). With walls = 1 the replica stays periodic along x and y;
 * along z it lies between a fixed wall at z = 0 and a wall at
 * z_w(n) = L_z + wall_u n dt after step n (n the step counter, dt that
 * step's dt; wall_u < 0 drives it in as a piston). No pair interacts across
 * the z boundary, and the SSA colours along z are those of a non-periodic
 * axis. A particle that crosses a wall during the drift is mirrored:
 * z -> 2 z_w - z and p_z -> 2 m u_w - p_z (u_w = 0 at z = 0). Positions
 * passed to dpde_set_state must lie in [0, z_w). A step after which the
 * moving wall would enter the lowest cell layer returns DPDE_ERR_ARG. */

/* Observables of one replica at the current state (Sec. II.B). */
typedef struct dpde_obs {
    double  E;           /* U + K + Eint                                    */
    double  K;           /* sum |p|^2 / (2m)                                */
    double  U;           /* potential energy                                */
    double  Eint;        /* sum eps_i                                       */
    double  P[3];        /* total momentum                                  */
    double  Tkin;        /* 2K / (d (n-1)), Eq. (Tkin), instantaneous       */
    double  Tint;        /* n / sum(C_v/eps_i), Eq. (Tint), instantaneous   */
    double  Tpot_num;    /* |grad U|^2 = sum |F_i|^2 (numerator of Eq. Tcon) */
    double  Tpot_den;    /* Laplacian of U (denominator of Eq. Tcon)        */
    int64_t step;        /* steps taken since dpde_set_state                */
    int64_t n;           /* particles in the replica                        */
    int64_t neg_eps;     /* number of eps_i <= 0                            */
    int64_t nonfinite;   /* number of particles with a NaN/Inf component    */
} dpde_obs;

typedef struct dpde_handle dpde_handle;

/* Creates a handle on the current CUDA device.
 *  params      : model parameters (copied).
 *  n_replicas  : >= 1.
 *  replicas    : n_replicas descriptors (copied). Every replica needs
 *                ncell_d = B_d floor(L_d/(B_d r_cut)) >= 3 and k_d >= 1.
 *  stream      : cudaStream_t to run on (NULL = legacy default stream). The
 *                caller keeps it alive for the handle's lifetime.
 *  out         : receives the handle (NULL on failure).
 * Allocates all device buffers for sum_r n_r particles. Errors: DPDE_ERR_ARG,
 * DPDE_ERR_OOM, DPDE_ERR_CUDA. */
int dpde_create(const dpde_params* params, int32_t n_replicas,
                const dpde_replica* replicas, void* stream, dpde_handle** out);

/* Sets the state of every replica and resets the step counter to `step`.
 *  q, p     : 3*N doubles, particle-major (x,y,z), replicas concatenated in
 *             order, ids = index within the replica's segment. q is wrapped
 *             into the box along periodic axes; along the z axis of a walled
 *             replica it is kept as given (z = L_z stays on the upper face).
 *             In DPDE_MIXED mode q, p are rounded to float.
 *  eps      : N doubles.
 *  on_device: 0 = host pointers, 1 = device pointers (e.g. torch data_ptr()).
 * Computes the forces F(q) of the new state. Synchronous. */
int dpde_set_state(dpde_handle* h, const double* q, const double* p,
                   const double* eps, int64_t step, int32_t on_device);

/* Copies the state out in id order (same layout as dpde_set_state); q in
 * [0, L) along periodic axes, between the walls along a walled z. Any of q,
 * p, eps may be NULL. Synchronous; returns the device
 * status (DPDE_ERR_NEG_EPS / DPDE_ERR_NONFINITE) raised since the last check. */
int dpde_get_state(dpde_handle* h, double* q, double* p, double* eps,
                   int32_t on_device);

/* Advances every replica by n >= 0 steps of size dt > 0 with the given scheme
 * (DPDE_SER, DPDE_HYBRID, DPDE_SEM, DPDE_SSA). Asynchronous on the handle's
 * stream; the returned status covers argument and launch errors. Device-side
 * conditions surface at the next dpde_sync / dpde_get_state /
 * dpde_observables. The step sequence is replayed from a captured CUDA graph
 * when use_graph != 0 (captured on first use per (dt, scheme)). */
int dpde_step(dpde_handle* h, int64_t n, double dt, int32_t scheme,
              int32_t use_graph);

/* Waits for the stream and returns the device status raised since the last
 * check (DPDE_OK, DPDE_ERR_NEG_EPS, DPDE_ERR_NONFINITE). */
int dpde_sync(dpde_handle* h);

/* Computes the observables of every replica into out[0 .. n_replicas-1].
 * Synchronous. Returns DPDE_ERR_NEG_EPS / _NONFINITE when the state holds
 * such values (out is still filled). */
int dpde_observables(dpde_handle* h, dpde_obs* out);

/* Raw checkpoint of the internal state (positions as cell + offset, momenta,
 * internal energies, forces, step counter) for a bit-exact restart.
 * dpde_checkpoint: with buf == NULL stores the required size in *size;
 * otherwise writes *size bytes to the host buffer buf. dpde_restore loads a
 * checkpoint made by a handle of identical parameters and replicas (checked:
 * DPDE_ERR_ARG otherwise). dpde_get_state / dpde_set_state round-trip
 * through absolute coordinates and are exact only to rounding. Synchronous. */
int dpde_checkpoint(dpde_handle* h, void* buf, uint64_t* size);
int dpde_restore(dpde_handle* h, const void* buf, uint64_t size);

/* Current step counter (steps since dpde_set_state plus its `step`). */
int dpde_get_step(dpde_handle* h, int64_t* step);

/* Frees the handle (NULL is accepted). */
int dpde_destroy(dpde_handle* h);

/* Last error message of the handle (or of the last failed dpde_create when h
 * is NULL). Never NULL; valid until the next call on the same handle. */
const char* dpde_last_error(const dpde_handle* h);

/* ---- observables without device allocation ---- */

/* Fixed limits of dpde_observables_noalloc (its scratch is one file-scope
 * device array of DPDE_NOALLOC_SCRATCH_BYTES = 4,217,344 bytes, about 4 MiB,
 * that every GPU which loads the library holds until the process exits). */
#define DPDE_NOALLOC_MAX_N            262144
#define DPDE_NOALLOC_MAX_CELLS        262144
#define DPDE_NOALLOC_SCRATCH_BYTES    4217344ull

/* Observables of one system (the quantities of dpde_observables, computed
 * in double) from a state the caller holds in device memory, without any
 * device allocation -- for callers that cannot call cudaMalloc: plug-ins
 * inside a host framework that owns all device memory through its own pool,
 * processes under a hard device-memory cap or with a no-allocation rule
 * after start-up. The paper has no counterpart; this is a service entry
 * point of the library, not part of the method.
 *  params  : m, r_cut, a of the system (sigma, seed, precision unused).
 *  replica : n <= DPDE_NOALLOC_MAX_N, box with floor(L_d / r_cut) >= 3 and
 *            prod_d floor(L_d / r_cut) <= DPDE_NOALLOC_MAX_CELLS, C_v
 *            (bricks unused). Larger systems: DPDE_ERR_ARG with a message
 *            from dpde_noalloc_last_error().
 *  q, p    : 3n doubles each, eps: n doubles -- DEVICE (or managed) pointers
 *            on the current device, read only; a host pointer or memory of
 *            another device is refused with DPDE_ERR_ARG before any launch.
 *            Along the z axis of a walled replica positions are not wrapped
 *            (z = 0 and z = L_z belong to the bottom and top cell layers).
 *  stream  : cudaStream_t to run on (NULL = legacy default stream).
 *  out     : one dpde_obs, host memory (out->step is 0).
 * All working memory is the library's fixed device scratch array; the call
 * clears the parts that must start at zero. The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) once for that device:
 * make it before any stream capture. Every call shares the array, so calls
 * whose work overlaps on a GPU race; callers serialise them. The call waits
 * for `stream` before returning. Returns DPDE_ERR_NEG_EPS / DPDE_ERR_NONFINITE
 * like dpde_observables (out is still filled; a pair with a non-finite
 * separation is skipped, as in the handle's pair search). */
int dpde_observables_noalloc(const dpde_params* params, const dpde_replica* replica,
                             const double* q, const double* p, const double* eps,
                             void* stream, dpde_obs* out);

/* Message of the last failed dpde_observables_noalloc call of this thread. */
const char* dpde_noalloc_last_error(void);

/* ---- diagnostics ---- */

/* Phases of one step, for dpde_step_profiled. */
#define DPDE_PHASE_KICK_DRIFT  0  /* Verlet first half, cell keys, counts  */
#define DPDE_PHASE_SCAN        1  /* prefix sum of the cell counts         */
#define DPDE_PHASE_GATHER      2  /* scatter + (cell, id) rank + gather    */
#define DPDE_PHASE_FORCE       3  /* forces + second half-kick             */
#define DPDE_PHASE_SSA         4  /* SSA chains (Hybrid set A, or SSA)      */
#define DPDE_PHASE_SWEEP1      5  /* SER first sweep                       */
#define DPDE_PHASE_SWEEP2      6  /* SER second sweep / SEM sweep / copy   */
#define DPDE_PHASE_OTHER       7  /* projection on the internal energies   */
#define DPDE_PHASE_SSA_GAUSS   8  /* SSA preparation: the pairs' Gaussians  */
                                  /* (ssa_mode 0, 1) or the level schedule  */
                                  /* (ssa_mode 2, whose execution draws the */
                                  /* Gaussians itself)                       */
#define DPDE_NUM_PHASES        9

/* Runs n steps like dpde_step without a graph, with CUDA events recorded on
 * the handle's stream around each phase; adds each phase's total elapsed
 * milliseconds over the n steps into phase_ms[DPDE_NUM_PHASES] (host array,
 * not cleared). Synchronous. */
int dpde_step_profiled(dpde_handle* h, int64_t n, double dt, int32_t scheme,
                       double* phase_ms);

/* ---- projection (Sec. IV.C) ---- */

/* Projection on the internal energies: with enable = 1, every later step
 * ends by lowering each eps_i of replica r by (E_r - E0[r]) / n_r, where E_r
 * is the total energy (U + K + sum eps) of the step's unconstrained update,
 * so that the total energy stays at E0[r]. E0: host array of n_replicas
 * doubles, or NULL for the handle's current energies (as dpde_observables
 * reports them). enable = 0 turns it off. Waits for the handle's stream and
 * drops the captured step graphs. The setting is not part of a checkpoint.
 * A step whose projection makes some eps_i <= 0 reports DPDE_ERR_NEG_EPS like
 * any other step. */
int dpde_set_projection(dpde_handle* h, int32_t enable, const double* E0);

/* ---- tuning ---- */

/* Launch parameters of a handle. None of them changes what is computed; the
 * tile edge changes the float rounding of pair separations in the force pass
 * (positions are shifted into a frame per tile), the block sizes change
 * nothing in the results. */
typedef struct dpde_tuning {
    int32_t tile_edge;   /* force tile edge in cells, 2..8 (default 6)                */
    int32_t block;       /* threads per block of the per-particle kernels: a multiple  */
                         /* of 32 in 64..1024 (default 256)                           */
    int32_t ssa_block;   /* threads per block of the per-class SSA launches and of the */
                         /* level form's execution: 32, 64, 96 or 128 (the per-domain  */
                         /* form runs one warp per block) (default 64)                */
    int32_t ssa_mode;    /* form of the SSA launches; all give the same results bit   */
                         /* for bit. 2 (default): by dependency levels -- per domain, */
                         /* every map of the sequence gets the level 1 + the larger   */
                         /* level of the last earlier maps of its two particles; a    */
                         /* block per domain runs the levels in order from shared     */
                         /* memory (maps of one level share no particle); used where  */
                         /* no domain is expected above 16,384 particles, else 0.     */
                         /* 0: one launch per colour class, a thread per cell;        */
                         /* 1 (Hybrid only, DPDE_SSA then takes 0): one launch in     */
                         /* which each warp takes whole domains and walks their       */
                         /* colour classes in order (domains share no chain, so their */
                         /* sequences commute), the domains' state staged in shared   */
                         /* memory where it fits; 3: the classes of mode 0 in one     */
                         /* persistent cooperative launch (a grid sized to full       */
                         /* co-residency), the blocks meeting at a grid barrier       */
                         /* between classes whose wait is bounded by the handle's     */
                         /* wait budget (dpde_set_wait_budget)                        */
    int32_t ssa_group;   /* domains per warp of ssa_mode 1, 1..8; 0 = automatic (32 /  */
                         /* the most cells of one class in one domain); get_tuning     */
                         /* reports the value in use                                   */
    int32_t reserved;    /* must be 0                                                  */
    double ms_per_step;  /* dpde_autotune: measured ms per step of the result; else 0  */
} dpde_tuning;

/* Wait budget of the grid barriers of the persistent SSA launch (ssa_mode
 * 3), in GPU clock cycles (default 2e9, about a second at 2 GHz): a block
 * that waits longer at a barrier raises a status and leaves, every other
 * block leaves at its next barrier, and the next dpde_sync returns
 * DPDE_ERR_TIMEOUT (the step's SSA part is then incomplete; set a state
 * again). 0 makes every block that has to wait give up at once. Waits for
 * the handle's stream and drops the captured step graphs. DPDE_ERR_ARG for
 * cycles < 0. */
int dpde_set_wait_budget(dpde_handle* h, int64_t cycles);

/* Current tuning of the handle (host pointer). */
int dpde_get_tuning(dpde_handle* h, dpde_tuning* out);

/* Sets the tuning (host pointer; ms_per_step ignored). Waits for the handle's
 * stream and drops the captured step graphs. DPDE_ERR_ARG for values outside
 * the ranges above. */
int dpde_set_tuning(dpde_handle* h, const dpde_tuning* t);

/* Autotuner: times `steps` graph-replayed steps of `scheme` at `dt` (after
 * one untimed replay) for each candidate -- tile edges 4..8, then per-particle block sizes
 * 128, 256, 512, then SSA block sizes 32, 64, 128, then the SSA modes 2, 1,
 * 0 and 3, then (Hybrid in ssa_mode 1) 1..4 domains per warp, each stage keeping the
 * best so far, a candidate replacing it only when more than 1% faster -- on
 * the handle's current state, restoring that state, its
 * forces and its step counter after every trial; then applies the fastest
 * tuning and writes it to *out (host pointer, may be NULL). The state after
 * the call equals the state before it. Synchronous. steps in 1..1000. */
int dpde_autotune(dpde_handle* h, int32_t scheme, double dt, int32_t steps, dpde_tuning* out);

/* Number of kernel launches in one step of `scheme` (the kernel nodes of
 * the step's CUDA graph, captured here without being run; *launches, host
 * pointer). The count depends on the handle's geometry and tuning: the SSA
 * part has three schedule launches (ssa_mode 2: the regular one and two for
 * domains beyond its capacities) and five execution launches (the regular
 * one, two for the domains it defers, two for those the schedule deferred,
 * the latter on a second stream beside the regular one), or one
 * launch drawing the Gaussians, then one per non-empty cell colour class
 * (ssa_mode 0, or DPDE_SSA in modes 1 and 2 without the level form), one
 * for all domains (Hybrid in ssa_mode 1) or one cooperative launch over all
 * classes (ssa_mode 3). No device work; the handle's state and step counter are
 * unchanged. DPDE_ERR_ARG for a bad scheme. */
int dpde_step_launches(dpde_handle* h, int32_t scheme, int64_t* launches);

/* Cell coordinates (cx, cy, cz) of every particle in id order (3N int32,
 * host pointer), as the library binned them at the end of the last step.
 * Synchronous. */
int dpde_get_cells(dpde_handle* h, int32_t* cells);

/* Runs the device Philox4x32-10 of the library on n (counter, key) pairs:
 * ctr is 4n uint32, key 2n uint32, out 4n uint32, all host pointers.
 * Used to check the device generator bit for bit. Synchronous. */
int dpde_debug_philox(int64_t n, const uint32_t* ctr, const uint32_t* key,
                      uint32_t* out);

/* Returns the library's device Gaussian triple G for n pairs
 * (seed, step, replica, id_a, id_b), with the sign convention G_ab = -G_ba:
 * out is 3n doubles (computed in double when precision = DPDE_FP64, in float
 * otherwise). Host pointers. Synchronous. */
int dpde_debug_gaussian(int64_t n, uint64_t seed, const uint32_t* step,
                        const uint32_t* replica, const uint32_t* id_a,
                        const uint32_t* id_b, int32_t precision, double* out);

#ifdef __cplusplus
}
#endif

#endif /* DPDE_H */
