// dpde_kernels.cuh -- the kernels of one DPDE timestep (templated on the
// precision T of positions, momenta, forces and pair arithmetic).
//
// Buffer roles are fixed per step so that one captured step graph can be
// replayed: the state lives in set A between steps; the cell sort gathers
// A -> B; forces and the FD schemes read B; the FD part writes the new state
// back into A (same cell-sorted slot order).
#pragma once

#include "dpde_device.cuh"

namespace dpde {

enum ListMode : int { LIST_NONE = 0, LIST_ALL = 1, LIST_CROSS = 2, LIST_FWD = 3 };

template <class T> struct Ctx {
    using vec = vec_t<T>;
    using E = eps_t<T>;
    vec* qA; vec* pA; E* eA; int* cA;
    vec* qB; vec* pB; E* eB; int* cB;
    uint32_t* idB;   // compact id copy of set B (for neighbour gathers)
    vec* F; vec* dp;
    T* upot;         // per particle: its share of U at the step's positions, 1/2 sum_j v(r_ij)
    int* key;        // global cell of each slot (A order), written by the drift
    int* tmp;        // slots binned by cell, arbitrary order inside a cell
    int* count;      // per-cell counts (ncells), followed by fill (ncells)
    int* fill;
    int* start;      // ncells + 1 exclusive prefix of count
    int* nbr_j;      // neighbour list, [k * N + i]
    T* nbr_w;        // 1 - r/r_cut of each entry
    int* nbr_n;      // entries per particle
    int nbr_cap;
    int* fwd_j;      // forward pairs of the SSA as the force pass writes them, entry-major
                     //   [k * N + i], partner slots in SSA sequence order (segment, id)
    T* fwd_w;        //   w = 1 - r/r_cut of each entry
    vec* fwd_g;      // (G_it, w) of each entry, particle-major [i * nbr_cap + k] (the SSA
                     //   chains' reading order), drawn before the SSA launches; the level
                     //   records of the SSA by levels; then the SER sweeps' delta p_ij
    int* fwd_n;
    const int* rep_of_slot;
    const int* rep_of_cell;
    const int* brick_rep;
    const int* tab;
    const RepInfo* reps;
    const long long* step;   // device step counter
    WallPos* wall;           // upper wall of each replica for this step's drift
    unsigned int* status;
    int N, ncells;
    T m, inv_m, rc, rc2, inv_rc, a, sigma, sig2_4;
    PotT<T> pot;
    uint2 seed;
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T texpm1(T x);
template <> __device__ __forceinline__ float texpm1(float x) { return expm1f(x); }
template <> __device__ __forceinline__ double texpm1(double x) { return expm1(x); }
template <class T> __device__ __forceinline__ T tfloor(T x);
template <> __device__ __forceinline__ float tfloor(float x) { return floorf(x); }
template <> __device__ __forceinline__ double tfloor(double x) { return floor(x); }

__device__ __forceinline__ float beta_of(ff e, const RepInfo& R) { return R.cvf / e.hi; }
__device__ __forceinline__ double beta_of(double e, const RepInfo& R) { return R.cv / e; }

__device__ __forceinline__ void flag(unsigned int* st, unsigned int bits) { atomicOr(st, bits); }

template <class V> __device__ __forceinline__ bool finite3(const V& v) {
    return isfinite(v.x) && isfinite(v.y) && isfinite(v.z);
}
__device__ __forceinline__ bool eps_ok(double e) { return e > 0.0; }
__device__ __forceinline__ bool eps_ok(ff e) { return e.hi > 0.0f; }
__device__ __forceinline__ bool eps_finite(double e) { return isfinite(e); }
__device__ __forceinline__ bool eps_finite(ff e) { return isfinite(e.hi) && isfinite(e.lo); }

template <class T>
__device__ __forceinline__ void check_state(unsigned int* st, const vec_t<T>& p, const eps_t<T>& e) {
    if (!eps_ok(e)) flag(st, ST_NEG_EPS);
    if (!finite3(p) || !eps_finite(e)) flag(st, ST_NONFINITE);
}

// offset * l for a cell offset d in {-1, 0, 1}
template <class T> __device__ __forceinline__ T shift(int d, T l) {
    return d == 0 ? T(0) : (d > 0 ? l : -l);
}

// Visits every particle j != i of the 27 cells around i's cell, in (dz, dy,
// x, slot) order, with the minimum-image separation q_i - q_j built from the
// cell offsets; body(j, qj, dx, dy, dz, r2, cross) is called for r2 < r_cut^2.
// cross tells whether j's cell lies in another brick than i's cell.
template <class T, class Body>
__device__ __forceinline__ void for_each_neighbour(const Ctx<T>& C, const vec_t<T>* __restrict__ q,
                                                   int i, const vec_t<T>& qi, int cc, const RepInfo& R,
                                                   Body&& body) {
    const int cx = cell_x(cc), cy = cell_y(cc), cz = cell_z(cc);
    const int nx = R.nc[0], ny = R.nc[1], nz = R.nc[2];
    const T lx = cell_len<T>(R, 0), ly = cell_len<T>(R, 1), lz = cell_len<T>(R, 2);
    const int* bt = brick_tab(C.tab, R);
    const int bx = __ldg(bt + cx), by = __ldg(bt + nx + cy), bz = __ldg(bt + nx + ny + cz);
    const int xm = cx == 0 ? nx - 1 : cx - 1;
    const int xp = cx == nx - 1 ? 0 : cx + 1;
    const bool xcross_m = __ldg(bt + xm) != bx, xcross_p = __ldg(bt + xp) != bx;
    for (int dz = -1; dz <= 1; ++dz) {
        int z = cz + dz;
        if (R.walls && (z < 0 || z >= nz)) continue;   // nothing beyond a wall
        z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
        const T sz = shift<T>(dz, lz);
        const bool zc = __ldg(bt + nx + ny + z) != bz;
        for (int dy = -1; dy <= 1; ++dy) {
            int y = cy + dy;
            y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
            const T sy = shift<T>(dy, ly);
            const bool rc = zc || (__ldg(bt + nx + y) != by);
            const int c0 = cell_index(C.tab, R, xm, y, z);
            const int c1 = cell_index(C.tab, R, cx, y, z);
            const int c2 = cell_index(C.tab, R, xp, y, z);
            auto visit_range = [&](int jb, int je, int dxc, bool cross) {
                const T sx = shift<T>(dxc, lx);
                for (int j = jb; j < je; ++j) {
                    if (j == i) continue;
                    const vec_t<T> qj = q[j];
                    const T ddx = (qi.x - qj.x) - sx;
                    const T ddy = (qi.y - qj.y) - sy;
                    const T ddz = (qi.z - qj.z) - sz;
                    const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                    if (r2 < C.rc2) body(j, qj, ddx, ddy, ddz, r2, cross);
                }
            };
            if (c1 == c0 + 1 && c2 == c1 + 1) {
                // the three x-cells are contiguous: one slot range
                const int b0 = C.start[c0], b1 = C.start[c1], b2 = C.start[c2], e = C.start[c2 + 1];
                visit_range(b0, b1, -1, rc || xcross_m);
                visit_range(b1, b2, 0, rc);
                visit_range(b2, e, 1, rc || xcross_p);
            } else {
                visit_range(C.start[c0], C.start[c0 + 1], -1, rc || xcross_m);
                visit_range(C.start[c1], C.start[c1 + 1], 0, rc);
                visit_range(C.start[c2], C.start[c2 + 1], 1, rc || xcross_p);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// state in / out
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_load_state(Ctx<T> C, const double* __restrict__ q, const double* __restrict__ p,
                             const double* __restrict__ e, int s0, int s1) {
    const int s = s0 + blockIdx.x * blockDim.x + threadIdx.x;   // slots s0 .. s1 - 1
    if (s >= s1) return;
    const RepInfo& R = C.reps[C.rep_of_slot[s]];
    vec_t<T> qv, pv;
    int c[3];
    T o[3];
    for (int d = 0; d < 3; ++d) {
        double x = q[3 * s + d];
        const bool wall = d == 2 && R.walls;   // a walled z is not periodic: z = L_z stays on the top face
        if (!wall && !(x >= 0.0 && x < R.L[d])) {   // wrap only what lies outside [0, L) (FP64 division is slow)
            x -= R.L[d] * floor(x / R.L[d]);
            if (x >= R.L[d]) x -= R.L[d];
        }
        int cd = (int)(x * R.s[d]);
        cd = cd > R.nc[d] - 1 ? R.nc[d] - 1 : (cd < 0 ? 0 : cd);
        c[d] = cd;
        o[d] = (T)(x - (double)cd * R.ell[d]);
    }
    qv.x = o[0]; qv.y = o[1]; qv.z = o[2];
    set_id(qv, (uint32_t)(s - R.part_off));
    eps_t<T> ev;
    eps_from(e[s], ev);
    pv.x = (T)p[3 * s]; pv.y = (T)p[3 * s + 1]; pv.z = (T)p[3 * s + 2];
    pv.w = beta_of(ev, R);
    C.qA[s] = qv;
    C.pA[s] = pv;
    C.eA[s] = ev;
    C.cA[s] = pack_cell(c[0], c[1], c[2]);
}

// slot of every particle of set A, by global id (part_off + id)
template <class T>
__global__ void k_slot_of_id(Ctx<T> C, int* __restrict__ slot_of) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.N) return;
    slot_of[C.reps[C.rep_of_slot[s]].part_off + (int)id_of(C.qA[s])] = s;
}

// the state of set A in id order: one thread per id gathers its slot, so the
// FP64 outputs are written contiguously
template <class T>
__global__ void k_get_state(Ctx<T> C, const int* __restrict__ slot_of, double* __restrict__ q,
                            double* __restrict__ p, double* __restrict__ e, int g0, int g1) {
    const int g = g0 + blockIdx.x * blockDim.x + threadIdx.x;   // ids g0 .. g1 - 1
    if (g >= g1) return;
    const int s = slot_of[g];
    const RepInfo& R = C.reps[C.rep_of_slot[s]];
    if (q) {
        const vec_t<T> qv = C.qA[s];
        const int cc = C.cA[s];
        const int cd[3] = {cell_x(cc), cell_y(cc), cell_z(cc)};
        const double od[3] = {(double)qv.x, (double)qv.y, (double)qv.z};
        for (int d = 0; d < 3; ++d) {
            double x = (double)cd[d] * R.ell[d] + od[d];
            if (!(d == 2 && R.walls)) {   // a walled z is not periodic
                if (x >= R.L[d]) x -= R.L[d];
                else if (x < 0.0) x += R.L[d];
            }
            q[3 * (size_t)g + d] = x;
        }
    }
    if (p) {
        const vec_t<T> pv = C.pA[s];
        p[3 * (size_t)g] = (double)pv.x; p[3 * (size_t)g + 1] = (double)pv.y; p[3 * (size_t)g + 2] = (double)pv.z;
    }
    if (e) e[g] = eps_value(C.eA[s]);
}

// ---------------------------------------------------------------------------
// Verlet first half: p += dt/2 F; q += dt p / m, with the offset moved into
// the neighbouring cell when it leaves [0, l) (periodic cell coordinates).
// Then the cell key and the per-cell count of the sort.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void move_axis(T& o, int& c, T l, int nc) {
    if (o >= l || o < T(0)) {
        const T f = tfloor(o / l);
        o -= f * l;
        c += (int)f;
        c %= nc;
        if (c < 0) c += nc;
    }
}

// Along a walled z axis: the drifted offset o of cell c, and its momentum
// p_z, mirrored at the wall z = 0 (z -> -z, p_z -> -p_z) or at the upper wall
// z_w = W.c l + W.o (z -> 2 z_w - z, p_z -> two_mu - p_z, two_mu = 2 m u),
// in cell-relative arithmetic.
template <class T>
__device__ __forceinline__ void wall_axis(T& o, int& c, T& pz, T l, int nc, const WallPos& W, T two_mu) {
    int cu = c;
    T on = o;
    if (on >= l || on < T(0)) {
        const T f = tfloor(on / l);
        on -= f * l;
        cu += (int)f;
        if (on >= l) { on -= l; ++cu; }
    }
    if (cu < 0) {
        cu = -cu - 1;
        on = l - on;
        if (on >= l) { on -= l; ++cu; }
        pz = -pz;
    } else {
        const T ow = (T)W.o;
        if (cu > W.c || (cu == W.c && on > ow)) {
            const T d = (T)(cu - W.c) * l + (on - ow);   // z - z_w > 0
            T o2 = ow - d;
            int c2 = W.c;
            const T f = tfloor(o2 / l);
            o2 -= f * l;
            c2 += (int)f;
            if (o2 >= l) { o2 -= l; ++c2; }
            cu = c2;
            on = o2;
            pz = two_mu - pz;
        }
    }
    // a position exactly on the upper face stays in the top cell
    if (cu >= nc) { cu = nc - 1; on = l; }
    if (cu < 0) { cu = 0; on = T(0); }
    o = on;
    c = cu;
}

// Upper-wall position of every replica for the drift of the current step n:
// z_w = L_z + u (n + 1) dt (L_z for replicas without walls). A wall inside
// the lowest cell layer raises ST_WALL.
template <class T>
__global__ void k_wall_pos(Ctx<T> C, int nrep, double dt) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrep) return;
    const RepInfo& I = C.reps[r];
    WallPos w;
    w.c = I.nc[2];
    w.o = 0.0;
    w.pad = 0;
    if (I.walls && I.wall_u != 0.0) {
        const double zw = I.L[2] + I.wall_u * (double)(*C.step + 1) * dt;
        int c = (int)floor(zw * I.s[2]);
        c = c > I.nc[2] ? I.nc[2] : c;
        double o = zw - (double)c * I.ell[2];
        if (o < 0.0) { --c; o += I.ell[2]; }
        if (c < 1) {
            flag(C.status, ST_WALL);
            c = 1;
            o = 0.0;
        }
        w.c = c;
        w.o = o;
    }
    C.wall[r] = w;
}

template <class T>
__global__ void k_kick_drift_key(Ctx<T> C, T half_dt, T dt, int kick) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.N) return;
    const int rep = C.rep_of_slot[s];
    const RepInfo& R = C.reps[rep];
    int cc = C.cA[s];
    int cx = cell_x(cc), cy = cell_y(cc), cz = cell_z(cc);
    if (kick) {
        vec_t<T> qv = C.qA[s];
        vec_t<T> pv = C.pA[s];
        const vec_t<T> f = C.F[s];
        pv.x += half_dt * f.x; pv.y += half_dt * f.y; pv.z += half_dt * f.z;
        const T c = dt * C.inv_m;
        qv.x += c * pv.x; qv.y += c * pv.y; qv.z += c * pv.z;
        move_axis(qv.x, cx, cell_len<T>(R, 0), R.nc[0]);
        move_axis(qv.y, cy, cell_len<T>(R, 1), R.nc[1]);
        if (R.walls)
            wall_axis(qv.z, cz, pv.z, cell_len<T>(R, 2), R.nc[2], C.wall[rep], T(2) * C.m * (T)R.wall_u);
        else
            move_axis(qv.z, cz, cell_len<T>(R, 2), R.nc[2]);
        cc = pack_cell(cx, cy, cz);
        C.pA[s] = pv;
        C.qA[s] = qv;
        C.cA[s] = cc;
    }
    const int key = cell_index(C.tab, R, cx, cy, cz);
    C.key[s] = key;
    atomicAdd(&C.count[key], 1);
}

// ---------------------------------------------------------------------------
// exclusive scan of the cell counts (three passes, 2048 elements per block)
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    const int warp_prefix = warp ? sh[warp - 1] : 0;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

__global__ void k_scan_local(const int* __restrict__ in, int* __restrict__ out, int* __restrict__ bsum,
                             int n) {
    __shared__ int sh[32];
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        sum += v[k];
    }
    int total;
    int run = block_exclusive_scan(sum, sh, total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void k_scan_bsums(int* __restrict__ bsum, int nb) {
    __shared__ int sh[32];
    int carry = 0;
    for (int t0 = 0; t0 < nb; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        const int v = t < nb ? bsum[t] : 0;
        int total;
        const int ex = block_exclusive_scan(v, sh, total);
        if (t < nb) bsum[t] = carry + ex;
        carry += total;
    }
}

__global__ void k_scan_add(int* __restrict__ out, const int* __restrict__ bsum, int n, int total) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[i / SCAN_TILE];
    if (i == 0) out[n] = total;
}

// ---------------------------------------------------------------------------
// counting sort by (cell, id): scatter into cells, then rank by id inside
// each cell and gather A -> B (refreshing beta = C_v / eps)
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_scatter(Ctx<T> C) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.N) return;
    const int c = C.key[s];
    C.tmp[C.start[c] + atomicAdd(&C.fill[c], 1)] = s;
}

template <class T>
__global__ void k_rank_gather(Ctx<T> C) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= C.N) return;
    const int s = C.tmp[t];
    const int c = C.key[s];
    const int b = C.start[c], e = C.start[c + 1];
    const vec_t<T> qv = C.qA[s];
    const uint32_t my = id_of(qv);
    int rank = 0;
    for (int u = b; u < e; ++u) rank += (id_of(C.qA[C.tmp[u]]) < my) ? 1 : 0;
    const int dst = b + rank;
    const RepInfo& R = C.reps[C.rep_of_slot[s]];
    vec_t<T> pv = C.pA[s];
    const eps_t<T> ev = C.eA[s];
    pv.w = beta_of(ev, R);
    C.qB[dst] = qv;
    C.pB[dst] = pv;
    C.eB[dst] = ev;
    C.cB[dst] = C.cA[s];
    C.idB[dst] = my;
}

// B -> A copy (after set_state and after the SSA-only scheme), refreshing beta
// and checking the state.
template <class T>
__global__ void k_copy_back(Ctx<T> C) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.N) return;
    const RepInfo& R = C.reps[C.rep_of_slot[s]];
    vec_t<T> pv = C.pB[s];
    const eps_t<T> ev = C.eB[s];
    pv.w = beta_of(ev, R);
    C.qA[s] = C.qB[s];
    C.pA[s] = pv;
    C.eA[s] = ev;
    C.cA[s] = C.cB[s];
    check_state<T>(C.status, pv, ev);
}

// ---------------------------------------------------------------------------
// conservative forces F(q) on B (soft repulsion a (1 - r/r_cut) r_hat), the
// second Verlet half-kick p += dt/2 F when kick != 0, and the lists of the
// fluctuation/dissipation part:
//   LIST_ALL   every neighbour (j, w = 1 - r/r_cut)           -> nbr
//   LIST_CROSS neighbours in another brick                      -> nbr
//              and forward neighbours in the same brick         -> fwd
//   LIST_FWD   forward neighbours (whole-replica SSA)           -> fwd
// A forward neighbour of i lies in the half stencil (segment > 13) or in
// i's own cell after i. Both force paths visit the neighbour cells in
// increasing segment s = 9 (dz+1) + 3 (dy+1) + (dx+1) and each cell in slot
// (= id) order, so a forward row lists i's pairs in SSA sequence order.
// ---------------------------------------------------------------------------
constexpr int NBR_J_BITS = 27;   // particle count limit 2^27 of a handle

template <class T> __device__ __forceinline__ T trsqrt(T x);
template <> __device__ __forceinline__ float trsqrt(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double trsqrt(double x) { return rsqrt(x); }

template <class T>
struct PairOut {
    T fx = 0, fy = 0, fz = 0;
    T u = 0;    // sum of v(r) over the neighbours
    int nn = 0, nf = 0;
};

// one neighbour j (global slot) of i at separation d with |d|^2 = r2; fwd
// tells whether j is a forward neighbour of i, cross whether j's brick
// differs from i's
template <class T, int LM>
__device__ __forceinline__ void force_hit(const Ctx<T>& C, int i, int j, bool fwd, bool cross, T dx, T dy, T dz,
                                          T r2, PairOut<T>& o) {
    const size_t N = (size_t)C.N;
    T w = T(1);
    if (r2 > T(0)) {
        const T ir = trsqrt(r2);
        w = T(1) - r2 * ir * C.inv_rc;
        T v, fr, lap;
        pair_pot(C.pot, r2, ir, v, fr, lap);
        o.fx += fr * dx; o.fy += fr * dy; o.fz += fr * dz;
        o.u += v;
    } else {
        o.u += pair_pot_at_zero(C.pot);
    }
    if (LM == LIST_ALL || (LM == LIST_CROSS && cross)) {
        if (o.nn < C.nbr_cap) {
            C.nbr_j[(size_t)o.nn * N + i] = j;
            C.nbr_w[(size_t)o.nn * N + i] = w;
        }
        ++o.nn;
    } else if ((LM == LIST_CROSS || LM == LIST_FWD) && fwd) {
        if (o.nf < C.nbr_cap) {
            const size_t at = (size_t)o.nf * N + i;
            C.fwd_j[at] = j;
            C.fwd_w[at] = w;
        }
        ++o.nf;
    }
}

template <class T, int LM>
__device__ __forceinline__ void force_finish(const Ctx<T>& C, int i, T half_dt, int kick, PairOut<T>& o) {
    if (o.nn > C.nbr_cap || o.nf > C.nbr_cap) {
        flag(C.status, ST_CAPACITY);
        o.nn = min(o.nn, C.nbr_cap);
        o.nf = min(o.nf, C.nbr_cap);
    }
    if (LM == LIST_ALL || LM == LIST_CROSS) C.nbr_n[i] = o.nn;
    if (LM == LIST_CROSS || LM == LIST_FWD) C.fwd_n[i] = o.nf;
    vec_t<T> f;
    f.x = o.fx; f.y = o.fy; f.z = o.fz; f.w = T(0);
    C.F[i] = f;
    // each pair is seen from both sides
    C.upot[i] = T(0.5) * o.u;
    if (kick) {
        vec_t<T> pv = C.pB[i];
        pv.x += half_dt * o.fx; pv.y += half_dt * o.fy; pv.z += half_dt * o.fz;
        C.pB[i] = pv;
    }
}

// Per-particle path on global memory (fallback for tiles whose halo does
// not fit in shared memory).
template <class T, int LM>
__device__ void force_one_global(const Ctx<T>& C, int i, T half_dt, int kick) {
    const RepInfo& R = C.reps[C.rep_of_slot[i]];
    const vec_t<T> qi = C.qB[i];
    const int cc = C.cB[i];
    const int cx = cell_x(cc), cy = cell_y(cc), cz = cell_z(cc);
    const int nx = R.nc[0], ny = R.nc[1], nz = R.nc[2];
    const T lx = cell_len<T>(R, 0), ly = cell_len<T>(R, 1), lz = cell_len<T>(R, 2);
    const int* bt = brick_tab(C.tab, R);
    const int bx = __ldg(bt + cx), by = __ldg(bt + nx + cy), bz = __ldg(bt + nx + ny + cz);
    PairOut<T> o;
    for (int sg = 0; sg < 27; ++sg) {
        const int dxc = sg % 3 - 1, dyc = (sg / 3) % 3 - 1, dzc = sg / 9 - 1;
        int x = cx + dxc, y = cy + dyc, z = cz + dzc;
        if (R.walls && (z < 0 || z >= nz)) continue;   // nothing beyond a wall
        x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
        y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
        z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
        const bool cross = __ldg(bt + x) != bx || __ldg(bt + nx + y) != by || __ldg(bt + nx + ny + z) != bz;
        const int c = cell_index(C.tab, R, x, y, z);
        const T sx = shift<T>(dxc, lx), sy = shift<T>(dyc, ly), sz = shift<T>(dzc, lz);
        const int e = C.start[c + 1];
        for (int j = C.start[c]; j < e; ++j) {
            if (j == i) continue;
            const vec_t<T> qj = C.qB[j];
            const T ddx = (qi.x - qj.x) - sx, ddy = (qi.y - qj.y) - sy, ddz = (qi.z - qj.z) - sz;
            const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
            if (r2 < C.rc2) force_hit<T, LM>(C, i, j, sg > 13 || (sg == 13 && j > i), cross, ddx, ddy, ddz, r2, o);
        }
    }
    force_finish<T, LM>(C, i, half_dt, kick, o);
}

// Tiled force pass: one block per tile of (up to) 6 x 6 x 6 cells. The tile
// and its one-cell halo are staged in shared memory in x-fastest halo-cell
// order (slot order inside a cell), with positions shifted into one frame
// centred on the tile, so a separation is a plain difference and the three
// x-cells of each (dy, dz) neighbour row of a particle form one contiguous
// range. In this layout j is a forward neighbour of i (later segment, or
// same cell and later slot) exactly when its halo index is larger, and the
// rows are visited in (segment, slot) order. The lanes of a warp walk the 9
// rows in step; the candidate loop only records hits (16-bit halo indices)
// in a per-thread shared buffer, and a second loop over the hits computes
// forces and lists -- so the costly part runs once per neighbour, not once
// per candidate of the slowest lane. Halos larger than hcap fall back to the
// global path.
constexpr int TILE_THREADS = 256;
constexpr int TILE_EDGE = 6;       // default tile edge (cells); the autotuner picks 4..8
constexpr int TILE_EDGE_MAX = 8;
constexpr int HIT_BUF = 28;        // hits buffered per thread (flushed when full)

// shared bytes before the staged particles, for halo cell capacity hcc
// ((edge + 2)^3): hstart, gstart, hbrick, rowoff (edge^2 + 1 <= 65), nown, hits
__host__ __device__ constexpr size_t tile_head_bytes(int hcc) {
    return ((size_t)(3 * hcc + 1 + 66) * sizeof(int) + (size_t)HIT_BUF * TILE_THREADS * 2 + 31) & ~(size_t)31;
}
// shared bytes per staged halo particle: position, global slot, brick, own
// index with its halo cell
template <class T>
__host__ __device__ constexpr size_t tile_per_particle() {
    return sizeof(vec_t<T>) + 2 * sizeof(int) + sizeof(unsigned int);
}

// One tile on the calling block. A tile whose halo holds more than hcap
// particles is appended to `defer` when that list is given (a second launch
// with a larger capacity takes it), else computed through the global path.
template <class T, int LM>
__device__ __forceinline__ void force_tile_run(const Ctx<T>& C, int tile, const int4* __restrict__ tile_org,
                                               const int4* __restrict__ tile_dim, T half_dt, int kick, int hcap,
                                               int hcc, int* defer, int* ndefer) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((size_t)smem_raw + 31) & ~(size_t)31);
    using vec = vec_t<T>;
    const int4 org = tile_org[tile];
    const int4 dim = tile_dim[tile];
    const RepInfo& R = C.reps[org.x];
    const int HX = dim.x + 2, HY = dim.y + 2, HZ = dim.z + 2;
    const int HC = HX * HY * HZ;
    const int nx = R.nc[0], ny = R.nc[1], nz = R.nc[2];
    // shared layout (sized for HC <= hcc = (edge + 2)^3):
    //   hstart[hcc+1] gstart[hcc] hbrick[hcc] rowoff[65] nown | hits[HIT_BUF][TILE_THREADS] (u16) |
    //   q[hcap] glob[hcap] brick[hcap] own[hcap] (u32: halo index | halo cell << 16)
    int* hstart = (int*)smem;
    int* gstart = hstart + hcc + 1;
    int* hbrick = gstart + hcc;
    int* rowoff = hbrick + hcc;
    int* nown = rowoff + 65;
    unsigned short* hits = (unsigned short*)(nown + 1);
    vec* hq = (vec*)(smem + tile_head_bytes(hcc));
    int* hglob = (int*)(hq + hcap);
    int* hbr = hglob + hcap;
    unsigned int* own = (unsigned int*)(hbr + hcap);   // halo index | halo cell << 16
    const int* bt = brick_tab(C.tab, R);
    // 1. halo cells: global start, count, brick (two cells per thread at a
    //    time, their loads issued together)
    for (int h0 = threadIdx.x; h0 < HC; h0 += 2 * blockDim.x) {
        int xs[2], ys[2], zs[2], cs[2];
        bool use[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int h = h0 + u * (int)blockDim.x;
            const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
            int x = org.y + hx - 1, y = org.z + hy - 1, z = org.w + hz - 1;
            use[u] = h < HC && !(R.walls && (z < 0 || z >= nz));   // beyond a wall: an empty halo cell
            x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
            y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
            z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
            xs[u] = x; ys[u] = y; zs[u] = z;
            cs[u] = use[u] ? cell_index(C.tab, R, x, y, z) : 0;
        }
        int a[2] = {0, 0}, b[2] = {0, 0}, br[2] = {-1, -1};
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (use[u]) {
                a[u] = C.start[cs[u]];
                b[u] = C.start[cs[u] + 1];
                br[u] = __ldg(bt + xs[u]) | (__ldg(bt + nx + ys[u]) << 10) | (__ldg(bt + nx + ny + zs[u]) << 20);
            }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int h = h0 + u * (int)blockDim.x;
            if (h < HC) {
                gstart[h] = a[u];
                hstart[h] = b[u] - a[u];
                hbrick[h] = br[u];
            }
        }
    }
    __syncthreads();
    // 2. exclusive scan of the halo counts (a run of up to 4 per thread, HC <= 1000)
    {
        __shared__ int sh[32];
        const int per = (HC + TILE_THREADS - 1) / TILE_THREADS;
        const int h0 = threadIdx.x * per;
        int v[4] = {0, 0, 0, 0}, run = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (u < per && h0 + u < HC) {
                v[u] = hstart[h0 + u];
                run += v[u];
            }
        int total;
        int ex = block_exclusive_scan(run, sh, total);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (u < per && h0 + u < HC) {
                hstart[h0 + u] = ex;
                ex += v[u];
            }
        if (threadIdx.x == 0) hstart[HC] = total;
    }
    __syncthreads();
    const int H = hstart[HC];
    const bool staged = H <= hcap;
    const T lx = cell_len<T>(R, 0), ly = cell_len<T>(R, 1), lz = cell_len<T>(R, 2);
    // 3. stage the halo particles (tile frame); 4. own-row offsets
    if (staged) {
        const int cxh = HX / 2, cyh = HY / 2, czh = HZ / 2;
        for (int h = threadIdx.x; h < HC; h += blockDim.x) {
            const int b = hstart[h], n = hstart[h + 1] - b, g = gstart[h];
            const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
            const T ox = (T)(hx - cxh) * lx, oy = (T)(hy - cyh) * ly, oz = (T)(hz - czh) * lz;
            const int br = hbrick[h];
            // four loads in flight at a time (a cell holds ~3 particles)
            for (int k0 = 0; k0 < n; k0 += 4) {
                vec qv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (k0 + u < n) qv[u] = C.qB[g + k0 + u];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (k0 + u < n) {
                        const int k = k0 + u;
                        qv[u].x += ox; qv[u].y += oy; qv[u].z += oz;
                        hq[b + k] = qv[u];
                        hglob[b + k] = g + k;
                        hbr[b + k] = br;
                    }
            }
        }
    }
    const int nrow = dim.y * dim.z;   // <= 64: a row per thread of the first two warps
    {
        __shared__ int s_w0;
        const int r = threadIdx.x;
        int v = 0;
        if (r < nrow) {
            const int h = ((r / dim.y + 1) * HY + (r % dim.y + 1)) * HX;
            v = hstart[h + dim.x + 1] - hstart[h + 1];
        }
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if ((r & 31) >= o) x += y;
        }
        if (r == 31) s_w0 = x;
        __syncthreads();
        if (r < nrow) {
            const int incl = x + (r >= 32 ? s_w0 : 0);
            rowoff[r] = incl - v;
            if (r == nrow - 1) {
                rowoff[nrow] = incl;
                *nown = incl;
            }
        }
    }
    __syncthreads();
    if (!staged) {
        if (defer) {
            if (threadIdx.x == 0) defer[atomicAdd(ndefer, 1)] = tile;
            return;
        }
        // fallback: own particles through the global path
        for (int r = threadIdx.x; r < nrow; r += blockDim.x) {
            const int h = ((r / dim.y + 1) * HY + (r % dim.y + 1)) * HX;
            for (int hc = h + 1; hc <= h + dim.x; ++hc) {
                const int g = gstart[hc], n = hstart[hc + 1] - hstart[hc];
                for (int k = 0; k < n; ++k) force_one_global<T, LM>(C, g + k, half_dt, kick);
            }
        }
        return;
    }
    // own particles in row order, a thread per own cell
    for (int rc = threadIdx.x; rc < nrow * dim.x; rc += blockDim.x) {
        const int r = rc / dim.x, cx = rc - r * dim.x;
        const int h = ((r / dim.y + 1) * HY + (r % dim.y + 1)) * HX;
        const int b = hstart[h + 1], k1 = hstart[h + cx + 2];
        const unsigned int cell = (unsigned int)(h + cx + 1) << 16;
        for (int k = hstart[h + cx + 1]; k < k1; ++k) own[rowoff[r] + (k - b)] = (unsigned int)k | cell;
    }
    __syncthreads();
    // 5. each own particle: rows in step, hits recorded, then processed
    const int no = *nown;
    unsigned short* myhits = hits + threadIdx.x;
    for (int k0 = 0; k0 < no; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        const bool act = k < no;
        const unsigned int ow = act ? own[k] : 0u;
        const int hi = (int)(ow & 0xffffu);
        const vec qi = hq[hi];
        const int i = hglob[hi];
        const int mybrick = hbr[hi];
        // i's halo cell, stored beside its halo index
        const int hc = (int)(ow >> 16);
        PairOut<T> o;
        int nh = 0;
        auto flush = [&]() {
            for (int u = 0; u < nh; ++u) {
                const int hj = myhits[u * TILE_THREADS];
                const vec qj = hq[hj];
                const T ddx = qi.x - qj.x, ddy = qi.y - qj.y, ddz = qi.z - qj.z;
                const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                force_hit<T, LM>(C, i, hglob[hj], hj > hi, hbr[hj] != mybrick, ddx, ddy, ddz, r2, o);
            }
            nh = 0;
        };
        auto near = [&](int j) {
            const vec qj = hq[j];
            const T ddx = qi.x - qj.x, ddy = qi.y - qj.y, ddz = qi.z - qj.z;
            return ddx * ddx + ddy * ddy + ddz * ddz < C.rc2 && j != hi;
        };
        for (int row = 0; row < 9; ++row) {
            const int base = hc + (row / 3 - 1) * HX * HY + (row % 3 - 1) * HX - 1;
            const int je = act ? hstart[base + 3] : 0;
            int j = act ? hstart[base] : 0;
            // four independent candidates per pass; every candidate is
            // written to the next free buffer slot and the slot kept only on
            // a hit (no branch per hit), so hits stay in order
            for (; j + 4 <= je; j += 4) {
                if (nh > HIT_BUF - 4) flush();
                const bool h0 = near(j), h1 = near(j + 1), h2 = near(j + 2), h3 = near(j + 3);
                myhits[nh * TILE_THREADS] = (unsigned short)j;
                nh += h0;
                myhits[nh * TILE_THREADS] = (unsigned short)(j + 1);
                nh += h1;
                myhits[nh * TILE_THREADS] = (unsigned short)(j + 2);
                nh += h2;
                myhits[nh * TILE_THREADS] = (unsigned short)(j + 3);
                nh += h3;
            }
            for (; j < je; ++j) {
                if (nh == HIT_BUF) flush();
                myhits[nh * TILE_THREADS] = (unsigned short)j;
                nh += near(j);
            }
        }
        flush();
        if (act) force_finish<T, LM>(C, i, half_dt, kick, o);
    }
}

template <class T, int LM>
__global__ void __launch_bounds__(TILE_THREADS) k_force_tile(Ctx<T> C, const int4* __restrict__ tile_org,
                                                             const int4* __restrict__ tile_dim, T half_dt,
                                                             int kick, int hcap, int hcc, int* defer,
                                                             int* ndefer) {
    force_tile_run<T, LM>(C, blockIdx.x, tile_org, tile_dim, half_dt, kick, hcap, hcc, defer, ndefer);
}

// The deferred tiles (dense regions), persistent blocks with a larger halo
// capacity; a tile beyond even that takes the global path.
template <class T, int LM>
__global__ void __launch_bounds__(TILE_THREADS) k_force_tile_dense(Ctx<T> C, const int4* __restrict__ tile_org,
                                                                   const int4* __restrict__ tile_dim, T half_dt,
                                                                   int kick, int hcap, int hcc,
                                                                   const int* __restrict__ defer,
                                                                   const int* __restrict__ ndefer) {
    const int n = *ndefer;
    for (int u = blockIdx.x; u < n; u += gridDim.x) {
        force_tile_run<T, LM>(C, defer[u], tile_org, tile_dim, half_dt, kick, hcap, hcc, nullptr, nullptr);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// SER (Sec. III.B.1) over the neighbour list.
// delta p_ij = -gamma_ij chi v_ij dt + sigma sqrt(chi) G_ij sqrt(dt),
// gamma_ij = sigma^2/4 (beta_i + beta_j) (Eq. DPDE_fd), chi = w^2.
//
// Both sweeps are warp-cooperative: a warp takes 32 consecutive particles
// (its lanes' own particles) and spreads all their list entries over its
// lanes, one entry per lane per pass, so every lane evaluates a pair on every
// pass however uneven the lists are. The pair values of one owner are summed
// by a segmented shuffle scan (in entry order inside a pass, passes in order:
// deterministic) and handed to the owner lane.
// ---------------------------------------------------------------------------
struct WarpEntries {
    int lane, nn, incl, total;
};

__device__ __forceinline__ WarpEntries warp_entries(int nn) {
    WarpEntries W;
    W.lane = threadIdx.x & 31;
    W.nn = nn;
    int incl = nn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (W.lane >= o) incl += y;
    }
    W.incl = incl;
    W.total = __shfl_sync(0xffffffffu, incl, 31);
    return W;
}

// owner lane of flat entry f (the first lane whose inclusive prefix exceeds f)
// and the entry's index k in the owner's list
__device__ __forceinline__ void warp_entry_owner(const WarpEntries& W, int f, int& owner, int& k) {
    int lo = 0;
#pragma unroll
    for (int st = 16; st > 0; st >>= 1) {
        const int v = __shfl_sync(0xffffffffu, W.incl, lo + st - 1);
        if (v <= f) lo += st;
    }
    owner = lo;
    k = f - __shfl_sync(0xffffffffu, W.incl - W.nn, lo);
}

// segmented sum of v over lanes with equal owner; returns to every lane the
// sum over this pass's entries of its own particle (0 if none)
template <class T>
__device__ __forceinline__ T warp_owner_sum(const WarpEntries& W, int f0, int owner, T v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, v, o);
        const int oy = __shfl_up_sync(0xffffffffu, owner, o);
        if (W.lane >= o && oy == owner) v += y;
    }
    // my entries in this pass end at flat index incl - 1
    const int last = W.incl - 1 - f0;
    const bool mine = W.nn > 0 && last >= 0 && W.incl - W.nn < f0 + 32;
    const T s = __shfl_sync(0xffffffffu, v, min(max(last, 0), 31));
    return mine ? s : T(0);
}

// delta p_ij of list entry k of particle i (pair arithmetic of Eq. SER_p)
template <class T>
__device__ __forceinline__ T3<T> ser_dp(const Ctx<T>& C, int i, int k, uint32_t step, T dt, T sdt,
                                        const vec_t<T>& pi, uint32_t idi, int rep) {
    const int j = C.nbr_j[(size_t)k * C.N + i];
    const T w = C.nbr_w[(size_t)k * C.N + i];
    const vec_t<T> pj = C.pB[j];
    const T3<T> G = pair_gauss<T>(C.seed, step, (uint32_t)rep, idi, C.idB[j]);
    const T A = -(C.sig2_4 * (pi.w + pj.w)) * (w * w) * dt;
    const T Bn = sdt * w;
    return T3<T>{A * ((pi.x - pj.x) * C.inv_m) + Bn * G.x, A * ((pi.y - pj.y) * C.inv_m) + Bn * G.y,
                 A * ((pi.z - pj.z) * C.inv_m) + Bn * G.z};
}

// first sweep: delta p_i = sum_j delta p_ij (Eq. SER_p). Each delta p_ij is
// also written, entry-major like the list, into the forward-entry buffer
// fwd_g (free once the SSA part of the step is done), so that the second
// sweep reads it instead of drawing the pair's Gaussian again.
template <class T>
__global__ void k_ser_sweep1(Ctx<T> C, T dt, T sqrt_dt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int base = i - (int)(threadIdx.x & 31);
    const WarpEntries W = warp_entries(i < C.N ? C.nbr_n[i] : 0);
    const uint32_t step = (uint32_t)*C.step;
    const T sdt = C.sigma * sqrt_dt;
    T ax = 0, ay = 0, az = 0;
    for (int f0 = 0; f0 < W.total; f0 += 32) {
        const int f = f0 + W.lane;
        int o, k;
        warp_entry_owner(W, f, o, k);
        T3<T> d{0, 0, 0};
        if (f < W.total) {
            const int io = base + o;
            d = ser_dp(C, io, k, step, dt, sdt, C.pB[io], C.idB[io], C.rep_of_slot[io]);
            // kept for the second sweep, entry-major like the list
            vec_t<T> dv;
            dv.x = d.x; dv.y = d.y; dv.z = d.z; dv.w = T(0);
            C.fwd_g[(size_t)k * C.N + io] = dv;
        } else {
            o = 32;
        }
        ax += warp_owner_sum(W, f0, o, d.x);
        ay += warp_owner_sum(W, f0, o, d.y);
        az += warp_owner_sum(W, f0, o, d.z);
    }
    if (i >= C.N) return;
    vec_t<T> out;
    out.x = ax; out.y = ay; out.z = az; out.w = T(0);
    C.dp[i] = out;
}

__device__ __forceinline__ double eps_half(double x) { return 0.5 * x; }
__device__ __forceinline__ ff eps_half(ff x) { return {0.5f * x.hi, 0.5f * x.lo}; }

// eps_i + add - Delta K_i, Delta K_i = (p' - p).(p' + p) / (2m) the kinetic-
// energy change of the stored momenta p -> p'. In FP64 plain arithmetic; in
// the mixed mode Delta K is formed as a compensated pair from exact
// two-sums and two-products of the float momenta, so that the internal
// energy absorbs the kinetic change to ~2^-46 relative rather than 2^-24.
__device__ __forceinline__ double eps_minus_dk(double e, double add, const d4& pn, const d4& pi, double hm) {
    const double dK = ((pn.x - pi.x) * (pn.x + pi.x) + (pn.y - pi.y) * (pn.y + pi.y) +
                       (pn.z - pi.z) * (pn.z + pi.z)) * hm;
    return e + (add - dK);
}
__device__ __forceinline__ ff eps_minus_dk(ff e, ff add, const float4& pn, const float4& pi, float hm) {
    float lx, ly, lz;
    const float hx = diff_of_squares(pn.x, pi.x, lx);
    const float hy = diff_of_squares(pn.y, pi.y, ly);
    const float hz = diff_of_squares(pn.z, pi.z, lz);
    float e1, e2;
    const float s1 = two_sum(hx, hy, e1);
    const float s2 = two_sum(s1, hz, e2);
    const float lo = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(lx, __fadd_rn(ly, lz)));
    // -Delta K as a pair (hm = 1/(2m), exact for a power-of-two mass)
    const float nh = -__fmul_rn(s2, hm), nl = -__fmul_rn(lo, hm);
    ff d;
    d.hi = __fadd_rn(nh, nl);
    d.lo = __fsub_rn(nl, __fsub_rn(d.hi, nh));
    return ff_add(ff_add(e, add), d);
}

// second sweep, Eq. (SER_eint_discretization), in the equivalent form
//   Delta eps_i = -Delta K_i + 1/2 sum_j T_ij,
//   T_ij = delta p_ij . (v_i + v_j + (delta p_i + delta p_j) / (2m)),
// where Delta K_i = (p_i' - p_i).(p_i' + p_i) / (2m) is the kinetic-energy
// change of the stored momenta. T_ij = -T_ji bit for bit, so the FD part
// conserves energy up to the rounding of per-particle sums. Writes the new
// state (q, cell, p, eps) into set A.
template <class T>
__global__ void k_ser_sweep2(Ctx<T> C, T dt, T sqrt_dt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int base = i - (int)(threadIdx.x & 31);
    const WarpEntries W = warp_entries(i < C.N ? C.nbr_n[i] : 0);
    const uint32_t step = (uint32_t)*C.step;
    const T sdt = C.sigma * sqrt_dt;
    const T hm = T(0.5) * C.inv_m;
    eps_t<T> tsum{};   // compensated in the mixed mode
    for (int f0 = 0; f0 < W.total; f0 += 32) {
        const int f = f0 + W.lane;
        int o, k;
        warp_entry_owner(W, f, o, k);
        T tv = 0;
        if (f < W.total) {
            const int io = base + o;
            const vec_t<T> pi = C.pB[io];
            const vec_t<T> dpi = C.dp[io];
            const int j = C.nbr_j[(size_t)k * C.N + io];
            const vec_t<T> d = C.fwd_g[(size_t)k * C.N + io];   // delta p_ij of the first sweep
            const vec_t<T> pj = C.pB[j];
            const vec_t<T> dpj = C.dp[j];
            const T vix = pi.x * C.inv_m, viy = pi.y * C.inv_m, viz = pi.z * C.inv_m;
            const T vjx = pj.x * C.inv_m, vjy = pj.y * C.inv_m, vjz = pj.z * C.inv_m;
            tv = d.x * ((vix + vjx) + (dpi.x + dpj.x) * hm) + d.y * ((viy + vjy) + (dpi.y + dpj.y) * hm) +
                 d.z * ((viz + vjz) + (dpi.z + dpj.z) * hm);
        } else {
            o = 32;
        }
        tsum = eps_add(tsum, warp_owner_sum(W, f0, o, tv));
    }
    if (i >= C.N) return;
    const RepInfo& R = C.reps[C.rep_of_slot[i]];
    const vec_t<T> pi = C.pB[i];
    const vec_t<T> dpi = C.dp[i];
    vec_t<T> pn = pi;
    pn.x = pi.x + dpi.x; pn.y = pi.y + dpi.y; pn.z = pi.z + dpi.z;
    const eps_t<T> en = eps_minus_dk(C.eB[i], eps_half(tsum), pn, pi, hm);
    pn.w = beta_of(en, R);
    C.qA[i] = C.qB[i];
    C.cA[i] = C.cB[i];
    C.pA[i] = pn;
    C.eA[i] = en;
    check_state<T>(C.status, pn, en);
}

// ---------------------------------------------------------------------------
// SEM, Eq. (SEM_fd): one sweep, Euler-Maruyama on p and eps. B -> A.
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_sem(Ctx<T> C, T dt, T sqrt_dt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.N) return;
    const int rep = C.rep_of_slot[i];
    const RepInfo& R = C.reps[rep];
    const vec_t<T> pi = C.pB[i];
    const uint32_t idi = C.idB[i];
    const uint32_t step = (uint32_t)*C.step;
    const int nn = C.nbr_n[i];
    const T d_sig2_m = T(3) * C.sigma * C.sigma * C.inv_m;
    const T sdt = C.sigma * sqrt_dt;
    T ax = 0, ay = 0, az = 0, de = 0;
    for (int k = 0; k < nn; ++k) {
        const int j = C.nbr_j[(size_t)k * C.N + i];
        const T w = C.nbr_w[(size_t)k * C.N + i];
        const vec_t<T> pj = C.pB[j];
        const T chi = w * w;
        const T gam = C.sig2_4 * (pi.w + pj.w);
        const T3<T> G = pair_gauss<T>(C.seed, step, (uint32_t)rep, idi, C.idB[j]);
        const T vx = (pi.x - pj.x) * C.inv_m;
        const T vy = (pi.y - pj.y) * C.inv_m;
        const T vz = (pi.z - pj.z) * C.inv_m;
        const T A = -gam * chi * dt, Bn = sdt * w;
        ax += A * vx + Bn * G.x;
        ay += A * vy + Bn * G.y;
        az += A * vz + Bn * G.z;
        de += T(0.5) * (gam * (vx * vx + vy * vy + vz * vz) - d_sig2_m) * chi * dt -
              T(0.5) * Bn * (vx * G.x + vy * G.y + vz * G.z);
    }
    vec_t<T> pn = pi;
    pn.x = pi.x + ax; pn.y = pi.y + ay; pn.z = pi.z + az;
    const eps_t<T> en = eps_add(C.eB[i], de);
    pn.w = beta_of(en, R);
    C.qA[i] = C.qB[i];
    C.cA[i] = C.cB[i];
    C.pA[i] = pn;
    C.eA[i] = en;
    check_state<T>(C.status, pn, en);
}

// ---------------------------------------------------------------------------
// SSA (Sec. III.A.2 and III.B.2): the pair map of Eq. (SSA_ij) -- the exact
// OU transition of p_st at fixed gamma_st, after which eps_s and eps_t each
// absorb -Delta K_st / 2 -- applied pair after pair in sequence order.
//
// The Gaussians do not depend on the state, so they are drawn first for every
// forward entry by a fully parallel pass (k_ssa_gauss) and stored with the
// entry's weight; the sequential part then only applies the maps.
//
// One launch per cell colour class; one thread per cell of the class. The
// cells reached by the pairs of two cells of one class are disjoint, so the
// threads touch disjoint particles and update set B in place. A thread walks
// its cell's chain -- the forward rows of the cell's particles s in slot
// (= id) order, concatenated -- as one flat loop, so the lanes of a warp
// diverge only by chain length. (p_s, eps_s, beta_s) stay in registers while
// s is current; the partner's updated (p_t, eps_t) goes back to memory at
// once, with beta_t = C_v / eps_t in p_t.w, so p.w is the current beta of
// every particle throughout. Partner indices are loaded two entries ahead,
// the partner state (and the next particle's state on a row change) one
// entry ahead. Loads issued ahead of a store can alias it only for the
// partner t being updated (two rows of a cell may share a partner, and a
// later particle of the cell may itself be t); those take the new values
// from registers.
// ---------------------------------------------------------------------------
constexpr int SSA_THREADS = 64;      // default block size; the autotuner picks 32..128
constexpr int SSA_THREADS_MAX = 128;
constexpr int SSA_ROWS = 20;     // rows per cell held in the shared row table
constexpr int NCOLOURS = 75;     // (2 + 1) x (3 + 2) x (3 + 2) cell colours

// G of every forward entry, with its weight: reads entry m of particle s at
// [m * N + s] (as the force pass wrote it) and writes (G_st, w)
// particle-major at [s * cap + m], the order the SSA chains read it. A
// warp takes 32 consecutive particles and spreads their entries over its
// lanes (a shuffle prefix sum of the row lengths gives each entry's owner).
template <class T>
__global__ void k_ssa_gauss(Ctx<T> C) {
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int base = s - lane;
    const int nf = s < C.N ? C.fwd_n[s] : 0;
    int incl = nf;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t step = (uint32_t)*C.step;
    const size_t cap = (size_t)C.nbr_cap;
    for (int f0 = 0; f0 < total; f0 += 32) {
        const int f = f0 + lane;
        // owner: the first lane whose inclusive prefix exceeds f
        int lo = 0;
#pragma unroll
        for (int step2 = 16; step2 > 0; step2 >>= 1) {
            const int v = __shfl_sync(0xffffffffu, incl, lo + step2 - 1);
            if (v <= f) lo += step2;
        }
        const int excl = __shfl_sync(0xffffffffu, incl - nf, lo);
        if (f < total) {
            const int so = base + lo;
            const size_t at = (size_t)(f - excl) * C.N + so;
            const size_t row = (size_t)so * cap + (f - excl);
            const int t = C.fwd_j[at];
            const T3<T> G = pair_gauss<T>(C.seed, step, (uint32_t)C.rep_of_slot[so], C.idB[so], C.idB[t]);
            vec_t<T> g;
            g.x = G.x; g.y = G.y; g.z = G.z; g.w = C.fwd_w[at];
            C.fwd_g[row] = g;
        }
    }
}

// The pair map on (p_s, eps_s, beta_s) in registers and partner (p_t, eps_t)
// with beta_t = p_t.w, for the entry (G, w) = g; returns the new partner
// state, beta in .w.
// beta = C_v / eps: exact in double; in float through the fast reciprocal
// (2 ulp), which keeps the chains' critical path short
__device__ __forceinline__ float ssa_beta(ff e, const RepInfo& R) { return __fdividef(R.cvf, e.hi); }
// sqrt(x / y) for x >= 0, y > 0: exact in double; in float x rsqrt(x y) (a
// few ulp, for x y a normal float; 0 for x = 0)
__device__ __forceinline__ float ssa_sqrt_ratio(float x, float y) {
    return x > 0.0f ? __fmul_rn(x, rsqrtf(__fmul_rn(x, y))) : 0.0f;
}
__device__ __forceinline__ double ssa_sqrt_ratio(double x, double y) { return sqrt(x / y); }
__device__ __forceinline__ double ssa_beta(double e, const RepInfo& R) { return R.cv / e; }

// Explicitly rounded operations: the compiler neither fuses nor reorders them,
// so every kernel that inlines the pair map computes the same bits.
__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float r_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double r_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// k2 = 2 dt / m
template <class T>
__device__ __forceinline__ void ssa_pair_map(const Ctx<T>& C, const RepInfo& R, vec_t<T>& ps, eps_t<T>& es,
                                             T& bs, vec_t<T>& pt, eps_t<T>& et, const vec_t<T>& g, T k2,
                                             T amp0) {
    const T w = g.w;
    const T chik = r_mul(r_mul(w, w), k2);
    const T gam = r_mul(C.sig2_4, r_add(bs, pt.w));
    const T aa = r_mul(gam, chik);   // a = 2 gamma chi dt / m
    // e^{-a} - 1, and 1 - e^{-2a} = -(e^{-a} - 1)(e^{-a} - 1 + 2)
    const T em1 = texpm1(-aa);
    const T x = r_mul(C.m, -r_mul(em1, r_add(em1, T(2))));   // m (1 - e^{-2a})
    const T amp = (gam != T(0)) ? r_mul(C.sigma, ssa_sqrt_ratio(x, gam)) : r_mul(amp0, w);
    const T Dx = r_mul(T(0.5), r_fma(em1, r_sub(ps.x, pt.x), r_mul(amp, g.x)));
    const T Dy = r_mul(T(0.5), r_fma(em1, r_sub(ps.y, pt.y), r_mul(amp, g.y)));
    const T Dz = r_mul(T(0.5), r_fma(em1, r_sub(ps.z, pt.z), r_mul(amp, g.z)));
    const T snx = r_add(ps.x, Dx), sny = r_add(ps.y, Dy), snz = r_add(ps.z, Dz);
    const T tnx = r_sub(pt.x, Dx), tny = r_sub(pt.y, Dy), tnz = r_sub(pt.z, Dz);
    // kinetic-energy change of the stored momenta, halved
    T q = r_mul(r_sub(tnz, pt.z), r_add(tnz, pt.z));
    q = r_fma(r_sub(tny, pt.y), r_add(tny, pt.y), q);
    q = r_fma(r_sub(tnx, pt.x), r_add(tnx, pt.x), q);
    q = r_fma(r_sub(snz, ps.z), r_add(snz, ps.z), q);
    q = r_fma(r_sub(sny, ps.y), r_add(sny, ps.y), q);
    q = r_fma(r_sub(snx, ps.x), r_add(snx, ps.x), q);
    const T dK = r_mul(q, r_mul(T(0.25), C.inv_m));
    ps.x = snx; ps.y = sny; ps.z = snz;
    es = eps_add(es, -dK);
    bs = ssa_beta(es, R);
    pt.x = tnx; pt.y = tny; pt.z = tnz;
    et = eps_add(et, -dK);
    pt.w = ssa_beta(et, R);
}

// Plain (unpipelined) chain, for cells with more than SSA_ROWS rows.
template <class T>
__device__ void ssa_chain_plain(const Ctx<T>& C, const RepInfo& R, int b, int e, T k2, T amp0) {
    const size_t cap = (size_t)C.nbr_cap;
    for (int s = b; s < e; ++s) {
        const int nf = C.fwd_n[s];
        if (nf == 0) continue;
        vec_t<T> ps = C.pB[s];
        eps_t<T> es = C.eB[s];
        T bs = ps.w;
        for (int m = 0; m < nf; ++m) {
            const int t = C.fwd_j[(size_t)m * C.N + s];
            const vec_t<T> g = C.fwd_g[(size_t)s * cap + m];
            vec_t<T> pt = C.pB[t];
            eps_t<T> et = C.eB[t];
            ssa_pair_map(C, R, ps, es, bs, pt, et, g, k2, amp0);
            C.pB[t] = pt;
            C.eB[t] = et;
        }
        ps.w = bs;
        C.pB[s] = ps;
        C.eB[s] = es;
    }
}

// dynamic shared memory of k_ssa_colour: two row tables [SSA_ROWS][block]
__host__ __device__ constexpr size_t ssa_smem_bytes(int block) { return (size_t)2 * SSA_ROWS * block * sizeof(int); }

// The chain of cell c on the calling thread (its column tid of the shared
// row tables, bdim columns).
template <class T>
__device__ __forceinline__ void ssa_cell_chain(const Ctx<T>& C, int c, T dt, T sqrt_dt, int* row_s, int* row_n,
                                               int bdim, int tid) {
    const int b = C.start[c], e = C.start[c + 1];
    int nrow = 0, total = 0;
    for (int s = b; s < e; ++s) {
        const int nf = C.fwd_n[s];
        if (nf > 0) {
            if (nrow < SSA_ROWS) {
                row_s[nrow * bdim + tid] = s;
                row_n[nrow * bdim + tid] = nf;
            }
            ++nrow;
            total += nf;
        }
    }
    if (total == 0) return;
    const RepInfo& R = C.reps[C.rep_of_cell[c]];
    const T amp0 = T(2) * C.sigma * sqrt_dt;   // amplitude of the map as gamma -> 0
    const T k2 = T(2) * dt * C.inv_m;
    if (nrow > SSA_ROWS) {
        ssa_chain_plain(C, R, b, e, k2, amp0);
        return;
    }
    const size_t cap = (size_t)C.nbr_cap;
    // position (r, m) of an entry; advancing past the last entry stays there
    auto advance = [&](int& r, int& m, int& nf) {
        if (m + 1 < nf) {
            ++m;
        } else if (r + 1 < nrow) {
            ++r;
            m = 0;
            nf = row_n[r * bdim + tid];
        }
    };
    // An entry of the chain: owner s, partner t, (G, w); the partner state,
    // and on a row switch the new owner's state, loaded two entries ahead.
    struct Ent {
        int s, t;
        vec_t<T> g, pt, ps;
        eps_t<T> et, es;
        bool sw;
    };
    auto load_index = [&](int r, int m, Ent& x) {
        x.s = row_s[r * bdim + tid];
        x.t = C.fwd_j[(size_t)m * C.N + x.s];
        x.g = C.fwd_g[(size_t)x.s * cap + m];
    };
    auto load_state = [&](Ent& x, int prev_s) {
        x.pt = C.pB[x.t];
        x.et = C.eB[x.t];
        x.sw = x.s != prev_s;
        if (x.sw) {
            x.ps = C.pB[x.s];
            x.es = C.eB[x.s];
        }
    };
    // the last two partner writes (w1 newest): the only stores a value loaded
    // two entries ahead can miss
    int w1t = -1, w2t = -1;
    vec_t<T> w1p, w2p;
    eps_t<T> w1e, w2e;
    auto patch = [&](int x, vec_t<T>& pv, eps_t<T>& ev) {
        if (x == w2t) { pv = w2p; ev = w2e; }
        if (x == w1t) { pv = w1p; ev = w1e; }
    };
    Ent e0, e1, e2;
    int r = 0, m = 0, nfr = row_n[tid];
    load_index(r, m, e0);
    load_state(e0, -1);
    advance(r, m, nfr);
    load_index(r, m, e1);
    load_state(e1, e0.s);
    advance(r, m, nfr);
    load_index(r, m, e2);
    int s = -1;
    vec_t<T> ps;
    eps_t<T> es;
    T bs = T(0);
    for (int k = 0; k < total; ++k) {
        // index of entry k + 3, state of entry k + 2
        advance(r, m, nfr);
        Ent e3;
        load_index(r, m, e3);
        load_state(e2, e1.s);
        // entry k becomes current: patch its loads with the writes they missed
        patch(e0.t, e0.pt, e0.et);
        if (e0.sw) {
            if (s >= 0) {
                ps.w = bs;
                C.pB[s] = ps;
                C.eB[s] = es;
            }
            patch(e0.s, e0.ps, e0.es);
            s = e0.s;
            ps = e0.ps;
            es = e0.es;
            bs = ps.w;
        }
        ssa_pair_map(C, R, ps, es, bs, e0.pt, e0.et, e0.g, k2, amp0);
        C.pB[e0.t] = e0.pt;
        C.eB[e0.t] = e0.et;
        w2t = w1t; w2p = w1p; w2e = w1e;
        w1t = e0.t; w1p = e0.pt; w1e = e0.et;
        e0 = e1;
        e1 = e2;
        e2 = e3;
    }
    ps.w = bs;
    C.pB[s] = ps;
    C.eB[s] = es;
}

// One colour class: one thread per cell of the class.
template <class T>
__global__ void __launch_bounds__(SSA_THREADS_MAX) k_ssa_colour(Ctx<T> C, const int* __restrict__ cells,
                                                                int ncol, T dt, T sqrt_dt) {
    extern __shared__ int ssa_rows[];
    const int bdim = blockDim.x;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= ncol) return;
    ssa_cell_chain(C, cells[u], dt, sqrt_dt, ssa_rows, ssa_rows + SSA_ROWS * bdim, bdim, (int)threadIdx.x);
}

// ---------------------------------------------------------------------------
// The same SSA sequence domain by domain (Hybrid, Sec. III.B.2). The chains of
// a domain never leave it, so two domains share no particle and their
// sequences commute: each warp takes `group` consecutive domains (one slot
// range, the cells being brick-major) and walks their colour classes in
// order, its lanes running the chains of one class at a time (cells of one
// class share no particle), with a warp barrier between classes (which also
// orders the lanes' memory accesses). The result is the class-by-class
// sequence bit for bit.
//
// The warp stages the state (p, eps) of its slot range in shared memory for
// all its classes when it fits in `scap` slots, and otherwise works on the
// state in place in global memory; in both cases a chain reads a state just
// before the map that uses it, so no load can miss an earlier store. The
// entries of a chain -- partner index and (G, w) -- are loaded SSA_AHEAD
// entries ahead. `bcells` holds the cells of each domain sorted by class,
// `boff[b * (NCOLOURS + 1) + k]` the start of class k of domain b and
// `bcell0[b]` the first cell of domain b (bcell0[nbricks] = ncells).
// ---------------------------------------------------------------------------
constexpr int SSA_GROUP_MAX = 8;
constexpr int SSA_AHEAD = 4;
constexpr int SSA_DOMAIN_SMEM = 200 * 1024;   // dynamic shared memory of one k_ssa_domains block, at most

// the particle state of a warp's slot range: staged (shared memory) or in place
template <class T>
struct SsaState {
    vec_t<T>* p;
    eps_t<T>* e;
    int base, n;   // slots base .. base + n - 1
};

// one forward entry of a chain: owner s, partner t, (G, w)
template <class T>
struct SsaEntry {
    int s, t;
    vec_t<T> g;
};

// next entry of the chain over slots .. e - 1 at (s, m) of a row of nf
// entries; false past the last
__device__ __forceinline__ bool ssa_next(const int* __restrict__ fwd_n, int& s, int& m, int& nf, int e) {
    if (m + 1 < nf) {
        ++m;
        return true;
    }
    for (++s; s < e; ++s) {
        nf = __ldg(fwd_n + s);
        if (nf > 0) {
            m = 0;
            return true;
        }
    }
    return false;
}

template <class T>
__device__ __forceinline__ bool ssa_fetch(const Ctx<T>& C, int& s, int& m, int& nf, int e, SsaEntry<T>& q) {
    if (!ssa_next(C.fwd_n, s, m, nf, e)) return false;
    q.s = s;
    q.t = __ldg(C.fwd_j + (size_t)m * C.N + s);
    q.g = C.fwd_g[(size_t)s * C.nbr_cap + m];
    return true;
}

// The chain of cell c on the state S. Entries are fetched in blocks of
// SSA_AHEAD into two register sets used in turn (the loop is unrolled over
// the pair, so no register is moved while its load is in flight): the loads
// of block i + 1 are issued before the maps of block i run.
template <class T>
__device__ __forceinline__ void ssa_domain_chain(const Ctx<T>& C, const RepInfo& R, int c, const SsaState<T>& S,
                                                 T k2, T amp0) {
    int s = C.start[c] - 1, m = 0, nf = 0;
    const int e = C.start[c + 1];
    int cur = -1;
    vec_t<T> ps;
    eps_t<T> es;
    T bs = T(0);
    bool bad = false;
    auto fill = [&](SsaEntry<T>(&q)[SSA_AHEAD], bool(&v)[SSA_AHEAD]) {
        bool more = true;
#pragma unroll
        for (int a = 0; a < SSA_AHEAD; ++a) {
            more = more && ssa_fetch(C, s, m, nf, e, q[a]);
            v[a] = more;
        }
    };
    auto run = [&](const SsaEntry<T>(&q)[SSA_AHEAD], const bool(&v)[SSA_AHEAD]) {
#pragma unroll
        for (int a = 0; a < SSA_AHEAD; ++a) {
            if (!v[a]) break;
            const SsaEntry<T>& x = q[a];
            const int ls = x.s - S.base, lt = x.t - S.base;
            if ((unsigned)ls >= (unsigned)S.n || (unsigned)lt >= (unsigned)S.n) {
                bad = true;   // a chain left its domain: never by construction
                break;
            }
            if (x.s != cur) {
                if (cur >= 0) {
                    ps.w = bs;
                    S.p[cur - S.base] = ps;
                    S.e[cur - S.base] = es;
                }
                cur = x.s;
                ps = S.p[ls];
                es = S.e[ls];
                bs = ps.w;
            }
            vec_t<T> pt = S.p[lt];
            eps_t<T> et = S.e[lt];
            ssa_pair_map(C, R, ps, es, bs, pt, et, x.g, k2, amp0);
            S.p[lt] = pt;
            S.e[lt] = et;
        }
    };
    SsaEntry<T> qa[SSA_AHEAD], qb[SSA_AHEAD];
    bool va[SSA_AHEAD], vb[SSA_AHEAD];
    fill(qa, va);
    while (va[0] && !bad) {
        fill(qb, vb);
        run(qa, va);
        if (!vb[0] || bad) break;
        fill(qa, va);
        run(qb, vb);
    }
    if (bad) {
        flag(C.status, ST_DOMAIN);
        return;
    }
    if (cur >= 0) {
        ps.w = bs;
        S.p[cur - S.base] = ps;
        S.e[cur - S.base] = es;
    }
}

// the colour classes of a warp's domains, in order, on the state S
template <class T>
__device__ __forceinline__ void ssa_domain_classes(const Ctx<T>& C, const int* __restrict__ bcells, const int* wo,
                                                   int nb, const SsaState<T>& S, T k2, T amp0) {
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < NCOLOURS; ++k) {
        int total = 0;
        for (int g = 0; g < nb; ++g) total += wo[g * (NCOLOURS + 1) + k + 1] - wo[g * (NCOLOURS + 1) + k];
        if (total == 0) continue;   // whole warp
        for (int i = lane; i < total; i += 32) {
            int g = 0, r = i;
            for (;;) {
                const int cnt = wo[g * (NCOLOURS + 1) + k + 1] - wo[g * (NCOLOURS + 1) + k];
                if (r < cnt) break;
                r -= cnt;
                ++g;
            }
            const int c = bcells[wo[g * (NCOLOURS + 1) + k] + r];
            ssa_domain_chain(C, C.reps[C.rep_of_cell[c]], c, S, k2, amp0);
        }
        __syncwarp();
    }
}

// shared memory of one warp of k_ssa_domains: staged p and eps for scap
// slots, then the class starts of `group` domains
template <class T>
__host__ __device__ constexpr size_t ssa_domain_warp_bytes(int group, int scap) {
    return (size_t)scap * (sizeof(vec_t<T>) + sizeof(eps_t<T>)) +
           (((size_t)group * (NCOLOURS + 1) * sizeof(int) + 15) / 16) * 16;
}

template <class T>
__global__ void __launch_bounds__(SSA_THREADS_MAX) k_ssa_domains(Ctx<T> C, const int* __restrict__ bcells,
                                                                 const int* __restrict__ boff,
                                                                 const int* __restrict__ bcell0, int nbricks,
                                                                 int group, int scap, T dt, T sqrt_dt) {
    extern __shared__ __align__(16) unsigned char ssa_dom_smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int b0 = (int)((blockIdx.x * (blockDim.x >> 5) + wib) * group);
    if (b0 >= nbricks) return;   // whole warp
    const int nb = min(group, nbricks - b0);
    unsigned char* wbase = ssa_dom_smem + (size_t)wib * ssa_domain_warp_bytes<T>(group, scap);
    int* wo = reinterpret_cast<int*>(wbase + (size_t)scap * (sizeof(vec_t<T>) + sizeof(eps_t<T>)));
    for (int i = lane; i < nb * (NCOLOURS + 1); i += 32) wo[i] = boff[(size_t)b0 * (NCOLOURS + 1) + i];
    const int sb = C.start[bcell0[b0]], se = C.start[bcell0[b0 + nb]];
    const T amp0 = T(2) * C.sigma * sqrt_dt;   // amplitude of the map as gamma -> 0
    const T k2 = T(2) * dt * C.inv_m;
    SsaState<T> S;
    S.base = sb;
    S.n = se - sb;
    if (S.n <= scap) {   // whole warp
        vec_t<T>* sp = reinterpret_cast<vec_t<T>*>(wbase);
        eps_t<T>* se_ = reinterpret_cast<eps_t<T>*>(wbase + (size_t)scap * sizeof(vec_t<T>));
        for (int i = lane; i < S.n; i += 32) {
            sp[i] = C.pB[sb + i];
            se_[i] = C.eB[sb + i];
        }
        __syncwarp();
        S.p = sp;
        S.e = se_;
        ssa_domain_classes(C, bcells, wo, nb, S, k2, amp0);
        __syncwarp();
        for (int i = lane; i < S.n; i += 32) {
            C.pB[sb + i] = sp[i];
            C.eB[sb + i] = se_[i];
        }
    } else {
        __syncwarp();
        S.p = C.pB + sb;
        S.e = C.eB + sb;
        ssa_domain_classes(C, bcells, wo, nb, S, k2, amp0);
    }
}

template <class T>
__global__ void k_refresh_beta(Ctx<T> C) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.N) return;
    C.pB[s].w = beta_of(C.eB[s], C.reps[C.rep_of_slot[s]]);
}

__global__ void k_step_inc(long long* step) { *step += 1; }

// ---------------------------------------------------------------------------
// Projection on the internal energies (Sec. IV.C): after the step, every
// eps_i of a replica is lowered by (E - E0)/N, E = U + K + sum eps of the
// unconstrained update (set A after the FD part; U from the force pass at the
// same positions). Per-chunk sums in a fixed order, then per replica.
// ---------------------------------------------------------------------------
constexpr int OBS_THREADS = 256;

template <class T>
__global__ void k_proj_chunks(Ctx<T> C, const int* __restrict__ chunk_begin, const int* __restrict__ chunk_end,
                              double* __restrict__ partial) {
    const int ch = blockIdx.x;
    double acc = 0.0;
    const double hm = 0.5 / (double)C.m;
    for (int i = chunk_begin[ch] + threadIdx.x; i < chunk_end[ch]; i += blockDim.x) {
        const vec_t<T> p = C.pA[i];
        acc += ((double)p.x * p.x + (double)p.y * p.y + (double)p.z * p.z) * hm + (double)C.upot[i] +
               eps_value(C.eA[i]);
    }
    __shared__ double sh[OBS_THREADS];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = OBS_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[ch] = sh[0];
}

template <class T>
__global__ void k_proj_reps(Ctx<T> C, const double* __restrict__ partial, const int* __restrict__ rep_chunk_begin,
                            int R, const double* __restrict__ E0, double* __restrict__ shift) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double E = 0.0;
    for (int ch = rep_chunk_begin[r]; ch < rep_chunk_begin[r + 1]; ++ch) E += partial[ch];
    const int n = C.reps[r].n;
    shift[r] = n > 0 ? (E - E0[r]) / (double)n : 0.0;
}

template <class T>
__global__ void k_proj_apply(Ctx<T> C, const double* __restrict__ shift) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.N) return;
    const int r = C.rep_of_slot[i];
    const eps_t<T> e = eps_add(C.eA[i], (T)(-shift[r]));
    C.eA[i] = e;
    vec_t<T> p = C.pA[i];
    p.w = beta_of(e, C.reps[r]);
    C.pA[i] = p;
    check_state<T>(C.status, p, e);
}

// ---------------------------------------------------------------------------
// observables: per-chunk sums (a chunk lies inside one replica), then per
// replica sums of the chunks in order -- deterministic.
// terms: 0 K, 1 U, 2 Eint, 3-5 P, 6 sum C_v/eps, 7 |F|^2, 8 Laplacian U,
//        9 neg eps, 10 nonfinite
// ---------------------------------------------------------------------------
constexpr int NTERMS = 11;

template <class T>
__global__ void k_obs_chunks(Ctx<T> C, const int* __restrict__ chunk_rep, const int* __restrict__ chunk_begin,
                             const int* __restrict__ chunk_end, double* __restrict__ partial) {
    const int ch = blockIdx.x;
    const int rep = chunk_rep[ch];
    const RepInfo& R = C.reps[rep];
    double acc[NTERMS];
    for (int k = 0; k < NTERMS; ++k) acc[k] = 0.0;
    for (int i = chunk_begin[ch] + threadIdx.x; i < chunk_end[ch]; i += blockDim.x) {
        const vec_t<T> qi = C.qA[i];
        const vec_t<T> pi = C.pA[i];
        const vec_t<T> f = C.F[i];
        const double e = eps_value(C.eA[i]);
        const bool fin = finite3(qi) && finite3(pi) && isfinite(e);
        acc[0] += ((double)pi.x * pi.x + (double)pi.y * pi.y + (double)pi.z * pi.z) * (0.5 / (double)C.m);
        acc[2] += e;
        acc[3] += pi.x; acc[4] += pi.y; acc[5] += pi.z;
        acc[6] += R.cv / e;
        acc[7] += (double)f.x * f.x + (double)f.y * f.y + (double)f.z * f.z;
        acc[9] += (e <= 0.0) ? 1.0 : 0.0;
        acc[10] += fin ? 0.0 : 1.0;
        if (fin) {
            // per neighbour, in the step's precision: v(r) and, for r > 0, the
            // Laplacian term v'' + 2 v'/r
            T usum = 0, lsum = 0;
            for_each_neighbour(C, C.qA, i, qi, C.cA[i], R,
                               [&](int, const vec_t<T>&, T, T, T, T r2, bool) {
                                   if (r2 > T(0)) {
                                       T v, fr, lap;
                                       pair_pot(C.pot, r2, trsqrt(r2), v, fr, lap);
                                       usum += v;
                                       lsum += lap;
                                   } else {
                                       usum += pair_pot_at_zero(C.pot);
                                   }
                               });
            acc[1] += 0.5 * (double)usum;   // each pair is seen twice
            acc[8] += (double)lsum;
        }
    }
    __shared__ double sh[NTERMS][OBS_THREADS];
    for (int k = 0; k < NTERMS; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = OBS_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < NTERMS; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < NTERMS) partial[(size_t)ch * NTERMS + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_obs_reps(const double* __restrict__ partial, const int* __restrict__ rep_chunk_begin,
                           int R, double* __restrict__ out) {
    const int r = blockIdx.x;
    if (r >= R || threadIdx.x >= NTERMS) return;
    double s = 0.0;
    for (int ch = rep_chunk_begin[r]; ch < rep_chunk_begin[r + 1]; ++ch) s += partial[(size_t)ch * NTERMS + threadIdx.x];
    out[(size_t)r * NTERMS + threadIdx.x] = s;
}

// cell coordinates of every particle in id order (diagnostic)
template <class T>
__global__ void k_get_cells(Ctx<T> C, int* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.N) return;
    const RepInfo& R = C.reps[C.rep_of_slot[s]];
    const long long g = (long long)R.part_off + id_of(C.qA[s]);
    const int cc = C.cA[s];
    out[3 * g] = cell_x(cc);
    out[3 * g + 1] = cell_y(cc);
    out[3 * g + 2] = cell_z(cc);
}

// ---------------------------------------------------------------------------
// diagnostics
// ---------------------------------------------------------------------------
__global__ void k_debug_philox(int n, const uint4* __restrict__ ctr, const uint2* __restrict__ key,
                               uint4* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], key[i]);
}

template <class T>
__global__ void k_debug_gauss(int n, uint2 seed, const uint32_t* __restrict__ step,
                              const uint32_t* __restrict__ rep, const uint32_t* __restrict__ a,
                              const uint32_t* __restrict__ b, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T3<T> g = pair_gauss<T>(seed, step[i], rep[i], a[i], b[i]);
    out[3 * i] = g.x; out[3 * i + 1] = g.y; out[3 * i + 2] = g.z;
}

}  // namespace dpde
