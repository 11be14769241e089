/*
 * oracle.c -- plain FP64 CPU reference of one DPDE timestep.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h): loaded by the tests, the smoke
 * check and the CPU baseline of the benchmark, never by the GPU library.
 *
 * Everything here is written for a reader checking it against the paper
 * (Homman, Maillet, Roussel, Stoltz, arXiv:1507.06643): one loop per formula,
 * no blocking or fusion, double precision throughout.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double ORA_TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11): a ten-round bijection of a 128-bit counter     */
/* under a 64-bit key. Each round multiplies words 0 and 2 by fixed odd     */
/* constants, keeps both halves of the 64-bit products, and mixes the high  */
/* halves into words 1 and 3 with the key; the key gets a Weyl increment    */
/* before every round but the first.                                         */
/* ------------------------------------------------------------------------ */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

void ora_philox_batch(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i) ora_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

/* G_ij^n of Sec. III.A (i.i.d. standard 3-d Gaussians with G_ji = -G_ij),
 * generated for the ordered pair (min id, max id) and negated for the other
 * orientation. Box-Muller on 24-bit uniforms. */
void ora_gaussian(uint64_t seed, uint32_t step, uint32_t replica, uint32_t id_a,
                  uint32_t id_b, double G[3])
{
    uint32_t lo = id_a < id_b ? id_a : id_b;
    uint32_t hi = id_a < id_b ? id_b : id_a;
    uint32_t ctr[4] = {lo, hi, step, replica};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t x[4];
    ora_philox4x32_10(ctr, key, x);
    double u1 = ((double)(x[0] >> 8) + 1.0) / 16777216.0;   /* (0, 1] */
    double t1 = (double)(x[1] >> 8) / 16777216.0;           /* [0, 1) */
    double u2 = ((double)(x[2] >> 8) + 1.0) / 16777216.0;
    double t2 = (double)(x[3] >> 8) / 16777216.0;
    double R1 = sqrt(-2.0 * log(u1));
    double R2 = sqrt(-2.0 * log(u2));
    double sign = (id_a <= id_b) ? 1.0 : -1.0;
    G[0] = sign * R1 * cos(ORA_TWO_PI * t1);
    G[1] = sign * R1 * sin(ORA_TWO_PI * t1);
    G[2] = sign * R2 * cos(ORA_TWO_PI * t2);
}

void ora_gaussian_batch(int64_t n, uint64_t seed, const uint32_t* step,
                        const uint32_t* replica, const uint32_t* id_a,
                        const uint32_t* id_b, double* out)
{
    for (int64_t i = 0; i < n; ++i)
        ora_gaussian(seed, step[i], replica[i], id_a[i], id_b[i], out + 3 * i);
}

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */

/* Whether axis d of a replica is periodic (z is not between walls). */
static int periodic_axis(const ora_replica* rep, int d) { return !(d == 2 && rep->walls); }

/* Minimum-image vector q_i - q_j (plain difference along a walled axis) and
 * its squared length. */
static double min_image(const ora_replica* rep, const double* q, int64_t i, int64_t j,
                        double dx[3])
{
    double r2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        double L = rep->box[d];
        double x = q[3 * i + d] - q[3 * j + d];
        if (periodic_axis(rep, d)) x -= L * round(x / L);
        dx[d] = x;
        r2 += x * x;
    }
    return r2;
}

int ora_cell_grid(const ora_replica* rep, double r_cut, int32_t* ncell, int32_t* k)
{
    for (int d = 0; d < 3; ++d) {
        if (rep->bricks[d] < 1) return -1;
        k[d] = (int32_t)floor(rep->box[d] / ((double)rep->bricks[d] * r_cut));
        ncell[d] = rep->bricks[d] * k[d];
        if (k[d] < 1 || ncell[d] < 3) return -1;
    }
    return 0;
}

/* c_d(x) = min(ncell_d - 1, (int)(x * (ncell_d / L_d))). */
static int cell_coord(double x, int32_t nc, double L)
{
    double s = (double)nc / L;
    int c = (int)(x * s);
    if (c > nc - 1) c = nc - 1;
    if (c < 0) c = 0;
    return c;
}

/* Particles of a replica binned by cell (z-major linear index), ascending
 * particle index (= id) inside each cell. */
typedef struct cell_list {
    int32_t nc[3], k[3];
    int64_t ncells;
    int64_t* start;   /* ncells + 1 */
    int64_t* member;  /* n */
    int32_t* coord;   /* 3n cell coordinates of each particle */
} cell_list;

static int build_cells(const ora_replica* rep, double r_cut, const double* q, cell_list* cl)
{
    if (ora_cell_grid(rep, r_cut, cl->nc, cl->k) != 0) return -1;
    int64_t n = rep->n;
    cl->ncells = (int64_t)cl->nc[0] * cl->nc[1] * cl->nc[2];
    cl->start = (int64_t*)calloc((size_t)cl->ncells + 1, sizeof(int64_t));
    cl->member = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    cl->coord = (int32_t*)malloc((size_t)(n > 0 ? 3 * n : 1) * sizeof(int32_t));
    int64_t* lin = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < 3; ++d) cl->coord[3 * i + d] = cell_coord(q[3 * i + d], cl->nc[d], rep->box[d]);
        lin[i] = ((int64_t)cl->coord[3 * i + 2] * cl->nc[1] + cl->coord[3 * i + 1]) * cl->nc[0] +
                 cl->coord[3 * i + 0];
        cl->start[lin[i] + 1] += 1;
    }
    for (int64_t c = 0; c < cl->ncells; ++c) cl->start[c + 1] += cl->start[c];
    int64_t* fill = (int64_t*)calloc((size_t)cl->ncells, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) cl->member[cl->start[lin[i]] + fill[lin[i]]++] = i;
    free(fill);
    free(lin);
    return 0;
}

static void free_cells(cell_list* cl)
{
    free(cl->start);
    free(cl->member);
    free(cl->coord);
}

int64_t ora_pairs_brute(const ora_replica* rep, double r_cut, const double* q, int64_t cap,
                        int64_t* pi, int64_t* pj)
{
    int64_t count = 0;
    double dx[3];
    for (int64_t i = 0; i < rep->n; ++i)
        for (int64_t j = i + 1; j < rep->n; ++j)
            if (min_image(rep, q, i, j, dx) < r_cut * r_cut) {
                if (pi && count < cap) { pi[count] = i; pj[count] = j; }
                ++count;
            }
    return count;
}

int64_t ora_pairs_cells(const ora_replica* rep, double r_cut, const double* q, int64_t cap,
                        int64_t* pi, int64_t* pj)
{
    cell_list cl;
    if (build_cells(rep, r_cut, q, &cl) != 0) return -1;
    int64_t count = 0;
    double dx[3];
    for (int64_t i = 0; i < rep->n; ++i) {
        const int32_t* ci = cl.coord + 3 * i;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int ddx = -1; ddx <= 1; ++ddx) {
                    if (!periodic_axis(rep, 2) && (ci[2] + dz < 0 || ci[2] + dz >= cl.nc[2])) continue;
                    int cx = (ci[0] + ddx + cl.nc[0]) % cl.nc[0];
                    int cy = (ci[1] + dy + cl.nc[1]) % cl.nc[1];
                    int cz = (ci[2] + dz + cl.nc[2]) % cl.nc[2];
                    int64_t c = ((int64_t)cz * cl.nc[1] + cy) * cl.nc[0] + cx;
                    for (int64_t s = cl.start[c]; s < cl.start[c + 1]; ++s) {
                        int64_t j = cl.member[s];
                        if (j <= i) continue;
                        if (min_image(rep, q, i, j, dx) < r_cut * r_cut) {
                            if (pi && count < cap) { pi[count] = i; pj[count] = j; }
                            ++count;
                        }
                    }
                }
    }
    free_cells(&cl);
    return count;
}

/* All interacting pairs (i < j) of a replica; brute force for small systems,
 * the cell list otherwise (the tests check that both give the same set). */
static int64_t all_pairs(const ora_replica* rep, double r_cut, const double* q, int64_t** pi,
                         int64_t** pj)
{
    int brute = rep->n < 512;
    int64_t np = brute ? ora_pairs_brute(rep, r_cut, q, 0, NULL, NULL)
                       : ora_pairs_cells(rep, r_cut, q, 0, NULL, NULL);
    if (np < 0) return -1;
    *pi = (int64_t*)malloc((size_t)(np > 0 ? np : 1) * sizeof(int64_t));
    *pj = (int64_t*)malloc((size_t)(np > 0 ? np : 1) * sizeof(int64_t));
    if (brute) ora_pairs_brute(rep, r_cut, q, np, *pi, *pj);
    else ora_pairs_cells(rep, r_cut, q, np, *pi, *pj);
    return np;
}

/* ------------------------------------------------------------------------ */
/* Conservative part                                                         */
/* ------------------------------------------------------------------------ */

/* F_i = -grad_{q_i} U with v(r) = (a r_cut/2)(1 - r/r_cut)^2, so the pair
 * force on i is a (1 - r/r_cut) (q_i - q_j)/r, and -(it) on j. */
/* Eq. (Ep): v = 4 eps_LJ((r_LJ/r)^12 - (r_LJ/r)^6) - eps_sh - f_sp (r - r_cut)
 * below r_cut, with eps_sh and f_sp fixed by v(r_cut) = 0 and v'(r_cut) = 0,
 * i.e. eps_sh = v_LJ(r_cut), f_sp = v_LJ'(r_cut). Soft repulsion otherwise. */
static void lj_terms(double eps, double rlj, double r, double* v, double* dv, double* d2v)
{
    double s6 = pow(rlj / r, 6.0), s12 = s6 * s6;
    *v = 4.0 * eps * (s12 - s6);
    *dv = 4.0 * eps * (-12.0 * s12 + 6.0 * s6) / r;
    *d2v = 4.0 * eps * (156.0 * s12 - 42.0 * s6) / (r * r);
}

void ora_pair_potential(const ora_params* prm, double r, double* v, double* dv, double* d2v)
{
    if (prm->potential == ORA_POT_LJ) {
        double vc, dvc, d2vc;
        lj_terms(prm->lj_eps, prm->lj_r, prm->r_cut, &vc, &dvc, &d2vc);
        lj_terms(prm->lj_eps, prm->lj_r, r, v, dv, d2v);
        *v -= vc + dvc * (r - prm->r_cut);
        *dv -= dvc;
        return;
    }
    double w = 1.0 - r / prm->r_cut;
    *v = 0.5 * prm->a * prm->r_cut * w * w;
    *dv = -prm->a * w;
    *d2v = prm->a / prm->r_cut;
}

int ora_forces(const ora_replica* rep, const ora_params* prm, const double* q, double* F)
{
    int64_t *pi, *pj;
    int64_t np = all_pairs(rep, prm->r_cut, q, &pi, &pj);
    if (np < 0) return -1;
    memset(F, 0, sizeof(double) * 3 * (size_t)rep->n);
    double dx[3];
    for (int64_t k = 0; k < np; ++k) {
        int64_t i = pi[k], j = pj[k];
        double r2 = min_image(rep, q, i, j, dx);
        double r = sqrt(r2);
        if (r == 0.0) continue;
        double v, dv, d2v;
        ora_pair_potential(prm, r, &v, &dv, &d2v);
        double f = -dv / r;   /* F_i = -v'(r) (q_i - q_j)/r */
        for (int d = 0; d < 3; ++d) {
            F[3 * i + d] += f * dx[d];
            F[3 * j + d] -= f * dx[d];
        }
    }
    free(pi);
    free(pj);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Fluctuation/dissipation pieces                                            */
/* ------------------------------------------------------------------------ */

typedef struct fd_ctx {
    const ora_replica* rep;
    const ora_params* prm;
    const double* q;
    double* p;
    double* eps;
    uint32_t step, ridx;
    double dt;
} fd_ctx;

static void pair_noise(const fd_ctx* c, int64_t i, int64_t j, double G[3])
{
    if (c->prm->noise)
        ora_gaussian(c->prm->seed, c->step, c->ridx, (uint32_t)i, (uint32_t)j, G);
    else
        G[0] = G[1] = G[2] = 0.0;
}

/* gamma_ij of Eq. (DPDE_fd) with T_i = eps_i / C_v. */
static double gamma_ij(const fd_ctx* c, int64_t i, int64_t j)
{
    double beta_i = c->rep->cv / c->eps[i];
    double beta_j = c->rep->cv / c->eps[j];
    return c->prm->sigma * c->prm->sigma / 4.0 * (beta_i + beta_j);
}

/* delta p_ij of Eq. (SER_p) (also the momentum increment of Eq. SEM_fd):
 * -gamma_ij chi v_ij dt + sigma sqrt(chi) G_ij sqrt(dt). */
static void pair_increment(const fd_ctx* c, int64_t i, int64_t j, double dpij[3])
{
    double dx[3];
    double r = sqrt(min_image(c->rep, c->q, i, j, dx));
    double w = 1.0 - r / c->prm->r_cut; /* sqrt(chi) */
    double chi = w * w;
    double g = gamma_ij(c, i, j);
    double G[3];
    pair_noise(c, i, j, G);
    for (int d = 0; d < 3; ++d) {
        double vij = (c->p[3 * i + d] - c->p[3 * j + d]) / c->prm->mass;
        dpij[d] = -g * chi * vij * c->dt + c->prm->sigma * w * G[d] * sqrt(c->dt);
    }
}

/* SER, Sec. III.B.1, over the given pairs: first sweep accumulates
 * delta p_i = sum_j delta p_ij (Eq. SER_p); second sweep
 * Delta eps_i = -1/2 sum_j delta p_ij . (v_ij + (delta p_i - delta p_j)/(2m))
 * (Eq. SER_eint_discretization); both sweeps read the pre-FD state, the
 * updates are applied at the end. */
static void ser_over_pairs(const fd_ctx* c, int64_t np, const int64_t* pi, const int64_t* pj)
{
    int64_t n = c->rep->n;
    double m = c->prm->mass;
    double* dp = (double*)calloc((size_t)(3 * n > 0 ? 3 * n : 1), sizeof(double));
    double* deps = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double* dpij = (double*)malloc((size_t)(np > 0 ? 3 * np : 1) * sizeof(double));
    for (int64_t k = 0; k < np; ++k) {
        int64_t i = pi[k], j = pj[k];
        pair_increment(c, i, j, dpij + 3 * k);
        for (int d = 0; d < 3; ++d) {
            dp[3 * i + d] += dpij[3 * k + d];
            dp[3 * j + d] -= dpij[3 * k + d]; /* delta p_ji = -delta p_ij */
        }
    }
    for (int64_t k = 0; k < np; ++k) {
        int64_t i = pi[k], j = pj[k];
        double ei = 0.0, ej = 0.0;
        for (int d = 0; d < 3; ++d) {
            double vij = (c->p[3 * i + d] - c->p[3 * j + d]) / m;
            double dij = dpij[3 * k + d];
            double dji = -dij;
            ei += dij * (vij + (dp[3 * i + d] - dp[3 * j + d]) / (2.0 * m));
            ej += dji * (-vij + (dp[3 * j + d] - dp[3 * i + d]) / (2.0 * m));
        }
        deps[i] += -0.5 * ei;
        deps[j] += -0.5 * ej;
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < 3; ++d) c->p[3 * i + d] += dp[3 * i + d];
        c->eps[i] += deps[i];
    }
    free(dp);
    free(deps);
    free(dpij);
}

/* SEM, Eq. (SEM_fd): Euler-Maruyama on p and eps from the pre-FD state. */
static void sem_over_pairs(const fd_ctx* c, int64_t np, const int64_t* pi, const int64_t* pj)
{
    int64_t n = c->rep->n;
    double m = c->prm->mass, sig = c->prm->sigma;
    double* dp = (double*)calloc((size_t)(3 * n > 0 ? 3 * n : 1), sizeof(double));
    double* deps = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    for (int64_t k = 0; k < np; ++k) {
        int64_t i = pi[k], j = pj[k];
        double dx[3], G[3], dpij[3];
        double r = sqrt(min_image(c->rep, c->q, i, j, dx));
        double w = 1.0 - r / c->prm->r_cut;
        double chi = w * w;
        double g = gamma_ij(c, i, j);
        pair_noise(c, i, j, G);
        double v2 = 0.0, vG = 0.0;
        for (int d = 0; d < 3; ++d) {
            double vij = (c->p[3 * i + d] - c->p[3 * j + d]) / m;
            dpij[d] = -g * chi * vij * c->dt + sig * w * G[d] * sqrt(c->dt);
            v2 += vij * vij;
            vG += vij * G[d];
        }
        for (int d = 0; d < 3; ++d) {
            dp[3 * i + d] += dpij[d];
            dp[3 * j + d] -= dpij[d];
        }
        /* the pair term is the same for i and j: v_ji = -v_ij, G_ji = -G_ij */
        double e = 0.5 * (g * v2 - 3.0 * sig * sig / m) * chi * c->dt - 0.5 * sig * w * vG * sqrt(c->dt);
        deps[i] += e;
        deps[j] += e;
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < 3; ++d) c->p[3 * i + d] += dp[3 * i + d];
        c->eps[i] += deps[i];
    }
    free(dp);
    free(deps);
}

/* One SSA pair map, Eq. (SSA_ij), in place: the exact Ornstein-Uhlenbeck
 * transition of p_ij = p_i - p_j at fixed gamma_ij (decay exponent
 * a = 2 gamma_ij chi dt / m), then eps_i, eps_j each absorb -Delta K_ij / 2. */
static void ssa_pair(const fd_ctx* c, int64_t i, int64_t j)
{
    double m = c->prm->mass, sig = c->prm->sigma;
    double dx[3], G[3];
    double r = sqrt(min_image(c->rep, c->q, i, j, dx));
    double w = 1.0 - r / c->prm->r_cut;
    double chi = w * w;
    double g = gamma_ij(c, i, j);
    double a = 2.0 * g * chi * c->dt / m;
    double amp = (g != 0.0) ? sig * sqrt(m * (-expm1(-2.0 * a)) / g) : 2.0 * sig * w * sqrt(c->dt);
    pair_noise(c, i, j, G);
    double K_before = 0.0, K_after = 0.0;
    double delta[3];
    for (int d = 0; d < 3; ++d) {
        double pij = c->p[3 * i + d] - c->p[3 * j + d];
        delta[d] = 0.5 * (expm1(-a) * pij + amp * G[d]);
        K_before += c->p[3 * i + d] * c->p[3 * i + d] + c->p[3 * j + d] * c->p[3 * j + d];
    }
    for (int d = 0; d < 3; ++d) {
        c->p[3 * i + d] += delta[d];
        c->p[3 * j + d] -= delta[d];
        K_after += c->p[3 * i + d] * c->p[3 * i + d] + c->p[3 * j + d] * c->p[3 * j + d];
    }
    double dK = (K_after - K_before) / (2.0 * m);
    c->eps[i] -= 0.5 * dK;
    c->eps[j] -= 0.5 * dK;
}

/* Colour of a cell coordinate l along one axis of a domain with k cells and
 * colour period P (3 along x and y, 2 along z -- the forward half stencil
 * spans offsets -1..1 along x and y but only 0..1 along z): l mod P, except
 * that along a periodic domain axis (one domain spanning a periodic axis of
 * the replica) the trailing k mod P cells take colours P, P + 1, so that two
 * cells of equal colour are at least P cells apart around the ring. */
static int axis_colour(int l, int k, int P, int periodic)
{
    int full = P * (k / P);
    if (periodic && l >= full) return P + (l - full);
    return l % P;
}

/* Enumerates the SSA sequence: visit(i, j) for each interacting pair of the
 * domain (Hybrid's set A: same brick; or the whole replica when whole_box),
 * in the order the library header defines: colours (cz, cy, cx) in
 * lexicographic order (z major); within a colour the cells are independent
 * (the cells their pairs reach are disjoint) and taken in any order; within a
 * cell, particles i by ascending id, each applying its forward pairs -- the
 * partners j in the 27 neighbour cells of the same domain whose cell offset
 * segment 9 (dz+1) + 3 (dy+1) + (dx+1) exceeds 13, or equals 13 (same cell)
 * with id_j > id_i -- ordered by (segment, id_j). */
typedef void (*pair_visitor)(void* ctx, int64_t i, int64_t j);

static int ssa_sequence(const ora_replica* rep, double r_cut, const double* q, int whole_box,
                        pair_visitor visit, void* ctx)
{
    cell_list cl;
    if (build_cells(rep, r_cut, q, &cl) != 0) return -1;
    int32_t B[3], k[3];
    for (int d = 0; d < 3; ++d) {
        B[d] = whole_box ? 1 : rep->bricks[d];
        k[d] = whole_box ? cl.nc[d] : cl.k[d];
    }
    double dx[3];
    const int period[3] = {3, 3, 2};
    for (int kz = 0; kz < 3; ++kz)
        for (int ky = 0; ky < 5; ++ky)
            for (int kx = 0; kx < 5; ++kx) {
                int kcol[3] = {kx, ky, kz};
                for (int cz = 0; cz < cl.nc[2]; ++cz)
                    for (int cy = 0; cy < cl.nc[1]; ++cy)
                        for (int cx = 0; cx < cl.nc[0]; ++cx) {
                            int cc[3] = {cx, cy, cz}, loc[3], brick[3];
                            int match = 1;
                            for (int d = 0; d < 3; ++d) {
                                loc[d] = cc[d] % k[d];
                                brick[d] = cc[d] / k[d];
                                const int ring = B[d] == 1 && periodic_axis(rep, d);
                                if (axis_colour(loc[d], k[d], period[d], ring) != kcol[d]) match = 0;
                            }
                            if (!match) continue;
                            int64_t c0 = ((int64_t)cz * cl.nc[1] + cy) * cl.nc[0] + cx;
                            for (int64_t si = cl.start[c0]; si < cl.start[c0 + 1]; ++si) {
                                int64_t i = cl.member[si];
                                for (int seg = 13; seg < 27; ++seg) {
                                    int del[3] = {seg % 3 - 1, (seg / 3) % 3 - 1, seg / 9 - 1};
                                    int nb[3], valid = 1;
                                    for (int d = 0; d < 3; ++d) {
                                        int ln = loc[d] + del[d];
                                        if (B[d] == 1 && periodic_axis(rep, d)) ln = (ln + k[d]) % k[d];
                                        else if (ln < 0 || ln >= k[d]) valid = 0;
                                        nb[d] = brick[d] * k[d] + ln;
                                    }
                                    if (!valid) continue;
                                    int64_t c1 = ((int64_t)nb[2] * cl.nc[1] + nb[1]) * cl.nc[0] + nb[0];
                                    for (int64_t t = cl.start[c1]; t < cl.start[c1 + 1]; ++t) {
                                        int64_t j = cl.member[t];
                                        if (seg == 13 && j <= i) continue;
                                        if (min_image(rep, q, i, j, dx) < r_cut * r_cut) visit(ctx, i, j);
                                    }
                                }
                            }
                        }
            }
    free_cells(&cl);
    return 0;
}

static void visit_ssa(void* ctx, int64_t i, int64_t j) { ssa_pair((const fd_ctx*)ctx, i, j); }

typedef struct order_sink { int64_t count, cap; int64_t *pi, *pj; } order_sink;
static void visit_record(void* ctx, int64_t i, int64_t j)
{
    order_sink* s = (order_sink*)ctx;
    if (s->pi && s->count < s->cap) { s->pi[s->count] = i; s->pj[s->count] = j; }
    s->count++;
}

int64_t ora_ssa_order(const ora_replica* rep, double r_cut, const double* q, int32_t whole_box,
                      int64_t cap, int64_t* pi, int64_t* pj)
{
    order_sink s = {0, cap, pi, pj};
    if (ssa_sequence(rep, r_cut, q, whole_box, visit_record, &s) != 0) return -1;
    return s.count;
}

/* Domain ("processor") index of particle i: brick_d = c_d / k_d. */
static int64_t brick_of(const ora_replica* rep, const int32_t* nc, const int32_t* k,
                        const double* q, int64_t i)
{
    int64_t b[3];
    for (int d = 0; d < 3; ++d) b[d] = cell_coord(q[3 * i + d], nc[d], rep->box[d]) / k[d];
    return (b[2] * rep->bricks[1] + b[1]) * rep->bricks[0] + b[0];
}

int ora_fd(const ora_replica* rep, int32_t ridx, const ora_params* prm, const double* q,
           double* p, double* eps, uint32_t step, double dt, int32_t scheme)
{
    fd_ctx c = {rep, prm, q, p, eps, step, (uint32_t)ridx, dt};
    int64_t *pi = NULL, *pj = NULL;
    int64_t np;
    switch (scheme) {
    case ORA_SER:
        np = all_pairs(rep, prm->r_cut, q, &pi, &pj);
        if (np < 0) return -1;
        ser_over_pairs(&c, np, pi, pj);
        break;
    case ORA_SEM:
        np = all_pairs(rep, prm->r_cut, q, &pi, &pj);
        if (np < 0) return -1;
        sem_over_pairs(&c, np, pi, pj);
        break;
    case ORA_SSA:
        if (ssa_sequence(rep, prm->r_cut, q, 1, visit_ssa, &c) != 0) return -1;
        break;
    case ORA_HYBRID: {
        /* Phi^Hybrid = Phi^{SER, A^c} o Phi^{SSA, i_l j_l} o ... o Phi^{SSA, i_1 j_1} */
        if (ssa_sequence(rep, prm->r_cut, q, 0, visit_ssa, &c) != 0) return -1;
        np = all_pairs(rep, prm->r_cut, q, &pi, &pj);
        if (np < 0) return -1;
        int32_t nc[3], k[3];
        ora_cell_grid(rep, prm->r_cut, nc, k);
        int64_t ncross = 0;
        for (int64_t t = 0; t < np; ++t)
            if (brick_of(rep, nc, k, q, pi[t]) != brick_of(rep, nc, k, q, pj[t])) {
                pi[ncross] = pi[t];
                pj[ncross] = pj[t];
                ++ncross;
            }
        ser_over_pairs(&c, ncross, pi, pj);
        break;
    }
    default:
        return -1;
    }
    free(pi);
    free(pj);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Full step: velocity Verlet, then the fluctuation/dissipation scheme       */
/* ------------------------------------------------------------------------ */

/* After the drift of step `step` (0-based): periodic wrap, or along a walled
 * z axis the specular reflections at z = 0 and at z_w = L_z + u (step + 1) dt
 * (z -> 2 z_w - z, p_z -> 2 m u - p_z). */
static void wrap_positions(const ora_replica* rep, const ora_params* prm, double* q, double* p,
                           int64_t step, double dt)
{
    const double zw = rep->box[2] + rep->wall_u * (double)(step + 1) * dt;
    for (int64_t i = 0; i < rep->n; ++i)
        for (int d = 0; d < 3; ++d) {
            double L = rep->box[d];
            double x = q[3 * i + d];
            if (!periodic_axis(rep, d)) {
                if (x < 0.0) {
                    x = -x;
                    p[3 * i + d] = -p[3 * i + d];
                } else if (x > zw) {
                    x = 2.0 * zw - x;
                    p[3 * i + d] = 2.0 * prm->mass * rep->wall_u - p[3 * i + d];
                }
            } else if (x >= L) {
                x -= L;
            } else if (x < 0.0) {
                x += L;
            }
            q[3 * i + d] = x;
        }
}

int ora_run(int32_t n_rep, const ora_replica* reps, const ora_params* prm, double* q,
            double* p, double* eps, double* F, int64_t step0, int64_t nsteps, double dt,
            int32_t scheme)
{
    if (n_rep < 1 || scheme < 0 || scheme > 3 || !(dt > 0.0)) return -1;
    int32_t nc[3], k[3];
    for (int r = 0; r < n_rep; ++r) {
        if (ora_cell_grid(&reps[r], prm->r_cut, nc, k) != 0) return -1;
        if (reps[r].walls != 0 && reps[r].walls != 1) return -1;
        if (reps[r].walls && !(reps[r].wall_u <= 0.0)) return -1;
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        int64_t off = 0;
        for (int r = 0; r < n_rep; ++r) {
            const ora_replica* rep = &reps[r];
            double* qr = q + 3 * off;
            double* pr = p + 3 * off;
            double* Fr = F + 3 * off;
            double* er = eps + off;
            int64_t n = rep->n;
            for (int64_t i = 0; i < 3 * n; ++i) pr[i] += 0.5 * dt * Fr[i];
            for (int64_t i = 0; i < 3 * n; ++i) qr[i] += dt * pr[i] / prm->mass;
            wrap_positions(rep, prm, qr, pr, step0 + s, dt);
            if (ora_forces(rep, prm, qr, Fr) != 0) return -1;
            for (int64_t i = 0; i < 3 * n; ++i) pr[i] += 0.5 * dt * Fr[i];
            if (ora_fd(rep, r, prm, qr, pr, er, (uint32_t)(step0 + s), dt, scheme) != 0) return -1;
            off += n;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Observables (Sec. II.B)                                                   */
/* ------------------------------------------------------------------------ */

int ora_observables(const ora_replica* rep, const ora_params* prm, const double* q,
                    const double* p, const double* eps, double* out)
{
    int64_t n = rep->n;
    double K = 0.0, Eint = 0.0, P[3] = {0, 0, 0}, inv_T = 0.0;
    int64_t neg = 0, bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        int finite = isfinite(eps[i]);
        for (int d = 0; d < 3; ++d) {
            K += p[3 * i + d] * p[3 * i + d] / (2.0 * prm->mass);
            P[d] += p[3 * i + d];
            finite = finite && isfinite(p[3 * i + d]) && isfinite(q[3 * i + d]);
        }
        Eint += eps[i];
        inv_T += rep->cv / eps[i];
        if (eps[i] <= 0.0) ++neg;
        if (!finite) ++bad;
    }
    double U = 0.0, lap = 0.0, gradsq = 0.0;
    if (bad == 0) {
        int64_t *pi, *pj;
        int64_t np = all_pairs(rep, prm->r_cut, q, &pi, &pj);
        if (np < 0) return -1;
        double dx[3];
        for (int64_t t = 0; t < np; ++t) {
            double r = sqrt(min_image(rep, q, pi[t], pj[t], dx));
            double v, dv, d2v;
            ora_pair_potential(prm, r, &v, &dv, &d2v);
            U += v;
            /* Laplacian of U: v'' + (d-1) v'/r, counted once for i and once for j */
            if (r > 0.0) lap += 2.0 * (d2v + 2.0 * dv / r);
        }
        free(pi);
        free(pj);
        double* F = (double*)malloc((size_t)(n > 0 ? 3 * n : 1) * sizeof(double));
        ora_forces(rep, prm, q, F);
        for (int64_t i = 0; i < 3 * n; ++i) gradsq += F[i] * F[i];
        free(F);
    }
    out[0] = U + K + Eint;
    out[1] = K;
    out[2] = U;
    out[3] = Eint;
    out[4] = P[0];
    out[5] = P[1];
    out[6] = P[2];
    out[7] = n > 1 ? 2.0 * K / (3.0 * (double)(n - 1)) : 0.0;
    out[8] = n > 0 ? (double)n / inv_T : 0.0;
    out[9] = gradsq;
    out[10] = lap;
    out[11] = (double)neg;
    out[12] = (double)bad;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Projection on the internal energies (Sec. IV.C): at the end of a step the */
/* internal energies of the unconstrained update are all lowered by          */
/* (E - E0) / N, E = U + K + sum eps of that update.                          */
/* ------------------------------------------------------------------------ */
int ora_project(const ora_replica* rep, const ora_params* prm, const double* q, const double* p,
                double* eps, double E0)
{
    double out[13];
    if (rep->n == 0) return 0;
    if (ora_observables(rep, prm, q, p, eps, out) != 0) return -1;
    double shift = (out[0] - E0) / (double)rep->n;
    for (int64_t i = 0; i < rep->n; ++i) eps[i] -= shift;
    return 0;
}
