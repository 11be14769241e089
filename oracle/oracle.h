/*
 * oracle.h -- plain, slow FP64 CPU reference ("oracle") of one DPDE timestep.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark may load this library. It shares no code with the
 * GPU library: it is written from the paper (Homman, Maillet, Roussel,
 * Stoltz, arXiv:1507.06643) and from the conventions it fixes below.
 *
 * Model (Sec. II.A): Eq. (DPDE) with chi of Eq. (pot_mou), the fluctuation/
 * dissipation relation Eq. (DPDE_fd), constant heat capacity eps = C_v T
 * (Eq. DPDE_internalEOS and Sec. IV.A), soft repulsion
 * v(r) = (a r_cut/2)(1 - r/r_cut)^2. Integrators (Sec. III): velocity Verlet
 * then one fluctuation/dissipation scheme: SEM Eq. (SEM_fd), SSA Eq.
 * (SSA_ij), SER Eqs. (SER_p), (SER_eint_discretization), Hybrid Sec. III.B.2.
 *
 * Conventions that the paper leaves open (noise generator, pair order of the
 * SSA sequence, cell grid, wrap) are the same definitions as the public
 * library header states; each is re-implemented here from that definition.
 *
 * Parity status: every function is pinned by the CPU tests (closed forms,
 * hand-worked cases, brute force, invariants) except ora_philox4x32_10's bit
 * pattern, which is pinned against cuRAND's Philox4x32-10 on a GPU machine.
 */
#ifndef DPDE_ORACLE_H
#define DPDE_ORACLE_H
#include <stdint.h>

typedef struct ora_params {
    double   mass, r_cut, a, sigma;
    uint64_t seed;
    int32_t  noise;     /* 1: Philox Gaussians; 0: G = 0 (tests only) */
    int32_t  potential; /* ORA_POT_SOFT or ORA_POT_LJ */
    double   lj_eps, lj_r;   /* Lennard-Jones eps_LJ and r_LJ (ORA_POT_LJ) */
} ora_params;

/* Pair potentials: the soft repulsion v = (a r_cut / 2)(1 - r/r_cut)^2, or the
 * shifted, splined and truncated Lennard-Jones potential of Eq. (Ep). */
enum { ORA_POT_SOFT = 0, ORA_POT_LJ = 1 };

/* v(r), v'(r), v''(r) of the pair potential (r < r_cut). */
void ora_pair_potential(const ora_params* prm, double r, double* v, double* dv, double* d2v);

/* A replica is periodic along x and y; along z it is periodic (walls = 0)
 * or closed by two specular walls (walls = 1): a fixed wall at z = 0 and a
 * wall at z_w(n) = L_z + wall_u n dt after step n (wall_u <= 0, a piston).
 * A particle that crosses a wall during the drift is reflected:
 * z -> 2 z_w - z, p_z -> 2 m u_w - p_z (u_w = 0 for the fixed wall), and no
 * pair interacts across the z boundary. This is the hard-wall reading of the
 * confining walls of the shock set-up (Sec. V). */
typedef struct ora_replica {
    int64_t n;
    double  box[3];
    double  cv;
    int32_t bricks[3];
    int32_t walls;
    double  wall_u;
} ora_replica;

enum { ORA_SER = 0, ORA_HYBRID = 1, ORA_SEM = 2, ORA_SSA = 3 };

/* Philox4x32-10 (Salmon et al., SC'11). */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void ora_philox_batch(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out);

/* Gaussian triple of pair (id_a, id_b) at step n of a replica, G_ab = -G_ba. */
void ora_gaussian(uint64_t seed, uint32_t step, uint32_t replica, uint32_t id_a,
                  uint32_t id_b, double G[3]);
void ora_gaussian_batch(int64_t n, uint64_t seed, const uint32_t* step,
                        const uint32_t* replica, const uint32_t* id_a,
                        const uint32_t* id_b, double* out);

/* Interacting pairs (i < j, r < r_cut) of one replica, by brute force over
 * all pairs or by a cell list. Returns the pair count; writes up to cap pairs
 * (sorted by (i, j)) to pi/pj when they are non-NULL. */
int64_t ora_pairs_brute(const ora_replica* rep, double r_cut, const double* q,
                        int64_t cap, int64_t* pi, int64_t* pj);
int64_t ora_pairs_cells(const ora_replica* rep, double r_cut, const double* q,
                        int64_t cap, int64_t* pi, int64_t* pj);

/* Conservative forces F(q) of one replica (3n doubles). */
int ora_forces(const ora_replica* rep, const ora_params* prm, const double* q, double* F);

/* Fluctuation/dissipation sub-step of one replica (replica index `ridx`, step
 * index `step` for the noise) on the given state, in place. */
int ora_fd(const ora_replica* rep, int32_t ridx, const ora_params* prm,
           const double* q, double* p, double* eps, uint32_t step, double dt,
           int32_t scheme);

/* Full timesteps of every replica (arrays concatenated by replica, 3n for q,
 * p, F and n for eps). F holds F(q) on entry and on exit. Returns 0, or -1 on
 * invalid arguments. */
int ora_run(int32_t n_rep, const ora_replica* reps, const ora_params* prm,
            double* q, double* p, double* eps, double* F, int64_t step0,
            int64_t nsteps, double dt, int32_t scheme);

/* Observables of one replica: out[0..12] = E, K, U, Eint, Px, Py, Pz, Tkin,
 * Tint, |grad U|^2, Laplacian U, neg_eps count, nonfinite count. */
int ora_observables(const ora_replica* rep, const ora_params* prm, const double* q,
                    const double* p, const double* eps, double* out);

/* Projection of Sec. IV.C on one replica, in place: eps_i -= (E - E0) / n,
 * E the total energy (U + K + sum eps) of the given state. */
int ora_project(const ora_replica* rep, const ora_params* prm, const double* q,
                const double* p, double* eps, double E0);

/* Cell grid of a replica as the library header defines it: ncell[3], k[3]. */
int ora_cell_grid(const ora_replica* rep, double r_cut, int32_t* ncell, int32_t* k);

/* SSA visiting order of a replica (Hybrid's set A, or every pair when
 * whole_box != 0): writes up to cap (i, j) pairs in sequence order; returns
 * the number of pairs. */
int64_t ora_ssa_order(const ora_replica* rep, double r_cut, const double* q,
                      int32_t whole_box, int64_t cap, int64_t* pi, int64_t* pj);

#endif
