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

enum ListMode : int { LIST_NONE = 0, LIST_ALL = 1, LIST_CROSS = 2 };

template <class T> struct Ctx {
    using vec = vec_t<T>;
    using E = eps_t<T>;
    vec* qA; vec* pA; E* eA; int* cA;
    vec* qB; vec* pB; E* eB; int* cB;
    uint32_t* idB;   // compact id copy of set B (for neighbour gathers)
    vec* F; vec* dp;
    int* key;        // global cell of each slot (A order), written by the drift
    int* tmp;        // slots binned by cell, arbitrary order inside a cell
    int* count;      // per-cell counts (ncells), followed by fill (ncells)
    int* fill;
    int* start;      // ncells + 1 exclusive prefix of count
    int* nbr_j;      // neighbour list, [k * N + i]
    T* nbr_w;        // 1 - r/r_cut of each entry
    int* nbr_n;      // entries per particle
    int nbr_cap;
    const int* rep_of_slot;
    const int* rep_of_cell;
    const int* brick_rep;
    const int* tab;
    const RepInfo* reps;
    const long long* step;   // device step counter
    unsigned int* status;
    int N, ncells;
    T m, inv_m, rc, rc2, inv_rc, a, sigma, sig2_4;
    uint2 seed;
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T tsqrt(T x);
template <> __device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
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
                             const double* __restrict__ e) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.N) return;
    const RepInfo& R = C.reps[C.rep_of_slot[s]];
    vec_t<T> qv, pv;
    int c[3];
    T o[3];
    for (int d = 0; d < 3; ++d) {
        double x = q[3 * s + d];
        x -= R.L[d] * floor(x / R.L[d]);
        if (x >= R.L[d]) x -= R.L[d];
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

template <class T>
__global__ void k_get_state(Ctx<T> C, double* __restrict__ q, double* __restrict__ p,
                            double* __restrict__ e) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.N) return;
    const RepInfo& R = C.reps[C.rep_of_slot[s]];
    const vec_t<T> qv = C.qA[s];
    const vec_t<T> pv = C.pA[s];
    const int cc = C.cA[s];
    const long long g = (long long)R.part_off + id_of(qv);
    if (q) {
        const int cd[3] = {cell_x(cc), cell_y(cc), cell_z(cc)};
        const double od[3] = {(double)qv.x, (double)qv.y, (double)qv.z};
        for (int d = 0; d < 3; ++d) {
            double x = (double)cd[d] * R.ell[d] + od[d];
            if (x >= R.L[d]) x -= R.L[d];
            else if (x < 0.0) x += R.L[d];
            q[3 * g + d] = x;
        }
    }
    if (p) { p[3 * g] = (double)pv.x; p[3 * g + 1] = (double)pv.y; p[3 * g + 2] = (double)pv.z; }
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

template <class T>
__global__ void k_kick_drift_key(Ctx<T> C, T half_dt, T dt, int kick) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.N) return;
    const RepInfo& R = C.reps[C.rep_of_slot[s]];
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
// second Verlet half-kick p += dt/2 F when kick != 0, and the neighbour list
// of the FD part (all pairs, or only cross-brick pairs for Hybrid's SER).
//
// Pass 1 walks the 27 neighbour cells as one flattened loop over 27 slot
// segments (so the lanes of a warp stay converged whatever the per-cell
// counts) and appends every particle within r_cut to the list, packed with
// its segment code. Pass 2 runs over these hits only (uniform trip counts):
// force, w = 1 - r/r_cut, and the final list (compacted to cross-brick
// entries for Hybrid). The two passes visit neighbours in the same order, so
// the force sums are deterministic.
// ---------------------------------------------------------------------------
constexpr int NBR_J_BITS = 27;   // slot index bits of a packed pass-1 entry
constexpr int NBR_J_MASK = (1 << NBR_J_BITS) - 1;

template <class T>
__global__ void __launch_bounds__(256) k_force(Ctx<T> C, T half_dt, int kick, int list_mode) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.N) return;
    const RepInfo& R = C.reps[C.rep_of_slot[i]];
    const vec_t<T> qi = C.qB[i];
    const int cc = C.cB[i];
    const int cx = cell_x(cc), cy = cell_y(cc), cz = cell_z(cc);
    const int nx = R.nc[0], ny = R.nc[1], nz = R.nc[2];
    const T lx = cell_len<T>(R, 0), ly = cell_len<T>(R, 1), lz = cell_len<T>(R, 2);
    const int* bt = brick_tab(C.tab, R);
    const int bx = __ldg(bt + cx), by = __ldg(bt + nx + cy), bz = __ldg(bt + nx + ny + cz);
    const int xm = cx == 0 ? nx - 1 : cx - 1;
    const int xp = cx == nx - 1 ? 0 : cx + 1;
    const bool xcm = __ldg(bt + xm) != bx, xcp = __ldg(bt + xp) != bx;
    // segment table: segment s = 9 (dz+1) + 3 (dy+1) + (dx+1)
    int sb[27], se[27];
    unsigned cross = 0;
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const int dz = r / 3 - 1, dy = r % 3 - 1;
        int z = cz + dz;
        z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
        int y = cy + dy;
        y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
        const bool rc = (__ldg(bt + nx + ny + z) != bz) || (__ldg(bt + nx + y) != by);
        const int c0 = cell_index(C.tab, R, xm, y, z);
        const int c1 = cell_index(C.tab, R, cx, y, z);
        const int c2 = cell_index(C.tab, R, xp, y, z);
        sb[3 * r] = C.start[c0];
        se[3 * r] = C.start[c0 + 1];
        sb[3 * r + 1] = C.start[c1];
        se[3 * r + 1] = C.start[c1 + 1];
        sb[3 * r + 2] = C.start[c2];
        se[3 * r + 2] = C.start[c2 + 1];
        cross |= (unsigned)(rc || xcm) << (3 * r);
        cross |= (unsigned)rc << (3 * r + 1);
        cross |= (unsigned)(rc || xcp) << (3 * r + 2);
    }
    // pass 1: candidates within r_cut -> packed (slot, segment) entries
    const size_t N = (size_t)C.N;
    int nh = 0;
    int seg = 0, j = sb[0], je = se[0];
    T sx = -lx, sy = -ly, sz = -lz;
    while (true) {
        while (j >= je) {
            if (++seg == 27) break;
            j = sb[seg];
            je = se[seg];
            const int dxs = seg % 3 - 1, dys = (seg / 3) % 3 - 1, dzs = seg / 9 - 1;
            sx = shift<T>(dxs, lx);
            sy = shift<T>(dys, ly);
            sz = shift<T>(dzs, lz);
        }
        if (seg == 27) break;
        if (j != i) {
            const vec_t<T> qj = C.qB[j];
            const T ddx = (qi.x - qj.x) - sx;
            const T ddy = (qi.y - qj.y) - sy;
            const T ddz = (qi.z - qj.z) - sz;
            const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
            if (r2 < C.rc2) {
                if (nh < C.nbr_cap) C.nbr_j[(size_t)nh * N + i] = j | (seg << NBR_J_BITS);
                ++nh;
            }
        }
        ++j;
    }
    if (nh > C.nbr_cap) {
        flag(C.status, ST_CAPACITY);
        nh = C.nbr_cap;
    }
    // pass 2: forces and the FD neighbour list
    T fx = 0, fy = 0, fz = 0;
    int nn = 0;
    for (int k = 0; k < nh; ++k) {
        const int packed = C.nbr_j[(size_t)k * N + i];
        const int jj = packed & NBR_J_MASK;
        const int sg = (int)((unsigned)packed >> NBR_J_BITS);
        const vec_t<T> qj = C.qB[jj];
        const T ddx = (qi.x - qj.x) - shift<T>(sg % 3 - 1, lx);
        const T ddy = (qi.y - qj.y) - shift<T>((sg / 3) % 3 - 1, ly);
        const T ddz = (qi.z - qj.z) - shift<T>(sg / 9 - 1, lz);
        const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
        const T r = tsqrt(r2);
        const T w = T(1) - r * C.inv_rc;
        if (r2 > T(0)) {
            const T f = C.a * w / r;
            fx += f * ddx; fy += f * ddy; fz += f * ddz;
        }
        if (list_mode == LIST_ALL || (list_mode == LIST_CROSS && ((cross >> sg) & 1u))) {
            C.nbr_j[(size_t)nn * N + i] = jj;
            C.nbr_w[(size_t)nn * N + i] = w;
            ++nn;
        }
    }
    if (list_mode != LIST_NONE) C.nbr_n[i] = nn;
    vec_t<T> f;
    f.x = fx; f.y = fy; f.z = fz; f.w = T(0);
    C.F[i] = f;
    if (kick) {
        vec_t<T> pv = C.pB[i];
        pv.x += half_dt * fx; pv.y += half_dt * fy; pv.z += half_dt * fz;
        C.pB[i] = pv;
    }
}

// ---------------------------------------------------------------------------
// SER (Sec. III.B.1) over the neighbour list.
// delta p_ij = -gamma_ij chi v_ij dt + sigma sqrt(chi) G_ij sqrt(dt),
// gamma_ij = sigma^2/4 (beta_i + beta_j) (Eq. DPDE_fd), chi = w^2.
// ---------------------------------------------------------------------------
// first sweep: delta p_i = sum_j delta p_ij (Eq. SER_p)
template <class T>
__global__ void k_ser_sweep1(Ctx<T> C, T dt, T sqrt_dt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.N) return;
    const int rep = C.rep_of_slot[i];
    const vec_t<T> pi = C.pB[i];
    const uint32_t idi = C.idB[i];
    const uint32_t step = (uint32_t)*C.step;
    const int nn = C.nbr_n[i];
    const T sdt = C.sigma * sqrt_dt;
    T ax = 0, ay = 0, az = 0;
    for (int k = 0; k < nn; ++k) {
        const int j = C.nbr_j[(size_t)k * C.N + i];
        const T w = C.nbr_w[(size_t)k * C.N + i];
        const vec_t<T> pj = C.pB[j];
        const T3<T> G = pair_gauss<T>(C.seed, step, (uint32_t)rep, idi, C.idB[j]);
        const T A = -(C.sig2_4 * (pi.w + pj.w)) * (w * w) * dt;
        const T Bn = sdt * w;
        ax += A * ((pi.x - pj.x) * C.inv_m) + Bn * G.x;
        ay += A * ((pi.y - pj.y) * C.inv_m) + Bn * G.y;
        az += A * ((pi.z - pj.z) * C.inv_m) + Bn * G.z;
    }
    vec_t<T> out;
    out.x = ax; out.y = ay; out.z = az; out.w = T(0);
    C.dp[i] = out;
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
    if (i >= C.N) return;
    const int rep = C.rep_of_slot[i];
    const RepInfo& R = C.reps[rep];
    const vec_t<T> pi = C.pB[i];
    const vec_t<T> dpi = C.dp[i];
    const uint32_t idi = C.idB[i];
    const uint32_t step = (uint32_t)*C.step;
    const int nn = C.nbr_n[i];
    const T sdt = C.sigma * sqrt_dt;
    const T hm = T(0.5) * C.inv_m;
    const T vix = pi.x * C.inv_m, viy = pi.y * C.inv_m, viz = pi.z * C.inv_m;
    T tsum = 0;
    for (int k = 0; k < nn; ++k) {
        const int j = C.nbr_j[(size_t)k * C.N + i];
        const T w = C.nbr_w[(size_t)k * C.N + i];
        const vec_t<T> pj = C.pB[j];
        const vec_t<T> dpj = C.dp[j];
        const T3<T> G = pair_gauss<T>(C.seed, step, (uint32_t)rep, idi, C.idB[j]);
        const T A = -(C.sig2_4 * (pi.w + pj.w)) * (w * w) * dt;
        const T Bn = sdt * w;
        const T vjx = pj.x * C.inv_m, vjy = pj.y * C.inv_m, vjz = pj.z * C.inv_m;
        const T dx = A * (vix - vjx) + Bn * G.x;
        const T dy = A * (viy - vjy) + Bn * G.y;
        const T dz = A * (viz - vjz) + Bn * G.z;
        tsum += dx * ((vix + vjx) + (dpi.x + dpj.x) * hm) + dy * ((viy + vjy) + (dpi.y + dpj.y) * hm) +
                dz * ((viz + vjz) + (dpi.z + dpj.z) * hm);
    }
    vec_t<T> pn = pi;
    pn.x = pi.x + dpi.x; pn.y = pi.y + dpi.y; pn.z = pi.z + dpi.z;
    const T dK = ((pn.x - pi.x) * (pn.x + pi.x) + (pn.y - pi.y) * (pn.y + pi.y) +
                  (pn.z - pi.z) * (pn.z + pi.z)) * hm;
    const eps_t<T> en = eps_add(C.eB[i], T(0.5) * tsum - dK);
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
// SSA pair map, Eq. (SSA_ij), on the pair (s, t) of the given arrays (shared
// or global memory): exact OU transition of p_st at fixed gamma_st, then
// eps_s, eps_t each absorb -Delta K_st / 2.
// ---------------------------------------------------------------------------
__constant__ int c_dirs[14][3] = {{0, 0, 0},   {1, 0, 0},  {-1, 1, 0}, {0, 1, 0},  {1, 1, 0},
                                  {-1, -1, 1}, {0, -1, 1}, {1, -1, 1}, {-1, 0, 1}, {0, 0, 1},
                                  {1, 0, 1},   {-1, 1, 1}, {0, 1, 1},  {1, 1, 1}};

// The state-dependent part of the SSA pair map, with w = 1 - r/r_cut and the
// Gaussian G_st already known.
template <class T>
__device__ __forceinline__ void ssa_apply(const Ctx<T>& C, const RepInfo& R, vec_t<T>* p, eps_t<T>* e,
                                          int s, int t, T w, T3<T> G, T dt, T sqrt_dt) {
    const vec_t<T> ps = p[s], pt = p[t];
    const eps_t<T> es = e[s], et = e[t];
    const T chi = w * w;
    const T gam = C.sig2_4 * (beta_of(es, R) + beta_of(et, R));
    const T a = T(2) * gam * chi * dt * C.inv_m;
    const T amp = (gam != T(0)) ? C.sigma * tsqrt(C.m * (-texpm1(T(-2) * a)) / gam)
                                : T(2) * C.sigma * w * sqrt_dt;
    const T em1 = texpm1(-a);
    const T Dx = T(0.5) * (em1 * (ps.x - pt.x) + amp * G.x);
    const T Dy = T(0.5) * (em1 * (ps.y - pt.y) + amp * G.y);
    const T Dz = T(0.5) * (em1 * (ps.z - pt.z) + amp * G.z);
    vec_t<T> sn = ps, tn = pt;
    sn.x = ps.x + Dx; sn.y = ps.y + Dy; sn.z = ps.z + Dz;
    tn.x = pt.x - Dx; tn.y = pt.y - Dy; tn.z = pt.z - Dz;
    // kinetic-energy change of the stored momenta, halved
    const T dK = ((sn.x - ps.x) * (sn.x + ps.x) + (sn.y - ps.y) * (sn.y + ps.y) +
                  (sn.z - ps.z) * (sn.z + ps.z) + (tn.x - pt.x) * (tn.x + pt.x) +
                  (tn.y - pt.y) * (tn.y + pt.y) + (tn.z - pt.z) * (tn.z + pt.z)) *
                 (T(0.25) * C.inv_m);
    p[s] = sn;
    p[t] = tn;
    e[s] = eps_add(es, -dK);
    e[t] = eps_add(et, -dK);
}

template <class T>
__device__ __forceinline__ void ssa_pair(const Ctx<T>& C, const RepInfo& R, uint32_t rep, uint32_t step,
                                         vec_t<T>* p, eps_t<T>* e, int s, int t, uint32_t ids,
                                         uint32_t idt, T r2, T dt, T sqrt_dt) {
    const T w = T(1) - tsqrt(r2) * C.inv_rc;
    ssa_apply(C, R, p, e, s, t, w, pair_gauss<T>(C.seed, step, rep, ids, idt), dt, sqrt_dt);
}

constexpr int SSA_THREADS = 256;

// One Hybrid domain ("brick") per block: the brick's particles (a contiguous
// slot range in brick-major cell order) are staged in shared memory when
// they fit (else the block works on global memory in place), then the SSA
// sequence runs round by round (14 directions x 2-3 colours). The cell
// pairs of a round touch disjoint particles. Each round has three phases:
//  (a) every cell pair lists its interacting pairs, in sequence order, into
//      a shared round buffer (w = 1 - r/r_cut);
//  (b) all lanes draw the Gaussians of the round's pairs;
//  (c) each cell pair applies its pair maps in order.
// A cell pair whose pairs do not fit in the buffer redoes its scan in (c)
// with inline Gaussians. Updates set B in place and refreshes beta.
template <class T>
__global__ void __launch_bounds__(SSA_THREADS) k_ssa_brick(Ctx<T> C, T dt, T sqrt_dt, int cap, int rcap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using vec = vec_t<T>;
    using E = eps_t<T>;
    // 32-byte aligned base (d4 vectors); the launch adds 32 bytes of slack
    unsigned char* smem = (unsigned char*)(((size_t)smem_raw + 31) & ~(size_t)31);
    const int g = blockIdx.x;
    const int rep = C.brick_rep[g];
    const RepInfo& R = C.reps[rep];
    const int kx = R.k[0], ky = R.k[1], kz = R.k[2];
    const int kc = kx * ky * kz;
    const int first = R.cell_off + (g - R.brick_off) * kc;
    const int base = C.start[first];
    const int cnt = C.start[first + kc] - base;
    // shared layout: rcount sst[kc+1] cbase[kc] ccnt[kc] | q[cap] p[cap] e[cap] |
    //                rs[rcap] rt[rcap] rw[rcap] rg[3 rcap]
    int& rcount = *(int*)smem;
    int* sst = (int*)smem + 1;
    int* cbase = sst + (kc + 1);
    int* ccnt = cbase + kc;
    size_t off = ((size_t)(3 * kc + 2) * sizeof(int) + 31) & ~(size_t)31;
    vec* sq = (vec*)(smem + off);
    vec* sp = sq + cap;
    E* se = (E*)(sp + cap);
    unsigned char* rb = (unsigned char*)(se + cap);
    rb = (unsigned char*)(((size_t)rb + 15) & ~(size_t)15);
    int* rs = (int*)rb;
    int* rt = rs + rcap;
    T* rw = (T*)(rt + rcap);
    T* rg = rw + rcap;
    const bool in_smem = cnt <= cap;
    for (int c = threadIdx.x; c <= kc; c += blockDim.x) sst[c] = C.start[first + c] - base;
    vec* q = in_smem ? sq : C.qB + base;
    vec* p = in_smem ? sp : C.pB + base;
    E* e = in_smem ? se : C.eB + base;
    if (in_smem)
        for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
            sq[s] = C.qB[base + s];
            sp[s] = C.pB[base + s];
            se[s] = C.eB[base + s];
        }
    if (threadIdx.x == 0) rcount = 0;
    __syncthreads();
    const uint32_t step = (uint32_t)*C.step;
    const T lx = cell_len<T>(R, 0), ly = cell_len<T>(R, 1), lz = cell_len<T>(R, 2);
    const int Bx = R.B[0], By = R.B[1], Bz = R.B[2];
    for (int di = 0; di < 14; ++di) {
        const int dxo = c_dirs[di][0], dyo = c_dirs[di][1], dzo = c_dirs[di][2];
        const int lead = dzo != 0 ? 2 : (dyo != 0 ? 1 : 0);
        const int klead = lead == 2 ? kz : (lead == 1 ? ky : kx);
        const int Blead = lead == 2 ? Bz : (lead == 1 ? By : Bx);
        const bool odd = (Blead == 1) && (klead & 1);
        // the (0,0,0) round is split in two halves by x parity: its cell
        // pairs are all disjoint, so any split keeps the sequence's meaning
        const int ncol = di == 0 ? 2 : (odd ? 3 : 2);
        const T sx = shift<T>(dxo, lx), sy = shift<T>(dyo, ly), sz = shift<T>(dzo, lz);
        for (int col = 0; col < ncol; ++col) {
            // (a) enumerate the round's pairs
            for (int c = threadIdx.x; c < kc; c += blockDim.x) {
                ccnt[c] = 0;
                const int lxc = c % kx, lyc = (c / kx) % ky, lzc = c / (kx * ky);
                if (di > 0) {
                    const int ll = lead == 2 ? lzc : (lead == 1 ? lyc : lxc);
                    const int my = (odd && ll == klead - 1) ? 2 : (ll & 1);
                    if (my != col) continue;
                } else if ((lxc & 1) != col) {
                    continue;
                }
                int nx = lxc + dxo, ny = lyc + dyo, nz = lzc + dzo;
                if (Bx == 1) nx = nx < 0 ? nx + kx : (nx >= kx ? nx - kx : nx);
                else if (nx < 0 || nx >= kx) continue;
                if (By == 1) ny = ny < 0 ? ny + ky : (ny >= ky ? ny - ky : ny);
                else if (ny < 0 || ny >= ky) continue;
                if (Bz == 1) nz = nz < 0 ? nz + kz : (nz >= kz ? nz - kz : nz);
                else if (nz < 0 || nz >= kz) continue;
                const int c1 = (nz * ky + ny) * kx + nx;
                const int e0 = sst[c + 1], e1 = sst[c1 + 1];
                int k = 0;
                for (int s = sst[c]; s < e0; ++s) {
                    const vec qs = q[s];
                    for (int t = (di == 0) ? s + 1 : sst[c1]; t < e1; ++t) {
                        const vec qt = q[t];
                        const T dx = (qs.x - qt.x) - sx, dy = (qs.y - qt.y) - sy, dz = (qs.z - qt.z) - sz;
                        k += (dx * dx + dy * dy + dz * dz < C.rc2) ? 1 : 0;
                    }
                }
                if (k == 0) continue;
                const int b = atomicAdd(&rcount, k);
                cbase[c] = b;
                ccnt[c] = (b + k <= rcap) ? k : -1;   // -1: redo inline in (c)
                if (b + k > rcap) {
                    // reserved slots below rcap stay unused: mark them
                    for (int m = b; m < rcap; ++m) rs[m] = -1;
                    continue;
                }
                int m = b;
                for (int s = sst[c]; s < e0; ++s) {
                    const vec qs = q[s];
                    for (int t = (di == 0) ? s + 1 : sst[c1]; t < e1; ++t) {
                        const vec qt = q[t];
                        const T dx = (qs.x - qt.x) - sx, dy = (qs.y - qt.y) - sy, dz = (qs.z - qt.z) - sz;
                        const T r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 < C.rc2) {
                            rs[m] = s;
                            rt[m] = t;
                            rw[m] = T(1) - tsqrt(r2) * C.inv_rc;
                            ++m;
                        }
                    }
                }
            }
            __syncthreads();
            // (b) Gaussians of the buffered pairs
            const int nr = min(rcount, rcap);
            for (int m = threadIdx.x; m < nr; m += blockDim.x) {
                const int s = rs[m], t = rt[m];
                if (s < 0 || s >= cnt || t < 0 || t >= cnt) continue;
                const T3<T> G = pair_gauss<T>(C.seed, step, (uint32_t)rep, id_of(q[s]), id_of(q[t]));
                rg[3 * m] = G.x;
                rg[3 * m + 1] = G.y;
                rg[3 * m + 2] = G.z;
            }
            __syncthreads();
            // (c) the pair maps, in sequence order within each cell pair
            for (int c = threadIdx.x; c < kc; c += blockDim.x) {
                const int k = ccnt[c];
                if (k > 0) {
                    for (int m = cbase[c]; m < cbase[c] + k; ++m)
                        ssa_apply(C, R, p, e, rs[m], rt[m], rw[m], T3<T>{rg[3 * m], rg[3 * m + 1], rg[3 * m + 2]},
                                  dt, sqrt_dt);
                } else if (k < 0) {
                    const int lxc = c % kx, lyc = (c / kx) % ky, lzc = c / (kx * ky);
                    int nx = lxc + dxo, ny = lyc + dyo, nz = lzc + dzo;
                    nx = nx < 0 ? nx + kx : (nx >= kx ? nx - kx : nx);
                    ny = ny < 0 ? ny + ky : (ny >= ky ? ny - ky : ny);
                    nz = nz < 0 ? nz + kz : (nz >= kz ? nz - kz : nz);
                    const int c1 = (nz * ky + ny) * kx + nx;
                    const int e0 = sst[c + 1], e1 = sst[c1 + 1];
                    for (int s = sst[c]; s < e0; ++s) {
                        const vec qs = q[s];
                        for (int t = (di == 0) ? s + 1 : sst[c1]; t < e1; ++t) {
                            const vec qt = q[t];
                            const T dx = (qs.x - qt.x) - sx, dy = (qs.y - qt.y) - sy, dz = (qs.z - qt.z) - sz;
                            const T r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 < C.rc2)
                                ssa_pair(C, R, (uint32_t)rep, step, p, e, s, t, id_of(qs), id_of(qt), r2, dt,
                                         sqrt_dt);
                        }
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) rcount = 0;
            __syncthreads();
        }
    }
    for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
        vec pv = p[s];
        pv.w = beta_of(e[s], R);
        C.pB[base + s] = pv;
        if (in_smem) C.eB[base + s] = e[s];
    }
}

// Whole-replica SSA (the DPDE_SSA scheme): one launch per (direction, colour)
// round over every cell of every replica, updating set B in place.
template <class T>
__global__ void k_ssa_round(Ctx<T> C, int di, int col, T dt, T sqrt_dt) {
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 >= C.ncells) return;
    const int rep = C.rep_of_cell[t0];
    const RepInfo& R = C.reps[rep];
    const int lc = t0 - R.cell_off;   // z-major enumeration of the replica's cells
    const int cc[3] = {lc % R.nc[0], (lc / R.nc[0]) % R.nc[1], lc / (R.nc[0] * R.nc[1])};
    const int* del = c_dirs[di];
    const int lead = del[2] != 0 ? 2 : (del[1] != 0 ? 1 : 0);
    if (di > 0) {
        const bool odd = R.nc[lead] & 1;
        const int ll = cc[lead];
        const int my = (odd && ll == R.nc[lead] - 1) ? 2 : (ll & 1);
        if (my != col) return;
    }
    int nb[3];
    for (int d = 0; d < 3; ++d) {
        int ln = cc[d] + del[d];
        nb[d] = ln < 0 ? ln + R.nc[d] : (ln >= R.nc[d] ? ln - R.nc[d] : ln);
    }
    const int c = cell_index(C.tab, R, cc[0], cc[1], cc[2]);
    const int c1 = cell_index(C.tab, R, nb[0], nb[1], nb[2]);
    const T sx = shift<T>(del[0], cell_len<T>(R, 0));
    const T sy = shift<T>(del[1], cell_len<T>(R, 1));
    const T sz = shift<T>(del[2], cell_len<T>(R, 2));
    const uint32_t step = (uint32_t)*C.step;
    const int e0 = C.start[c + 1], e1 = C.start[c1 + 1];
    for (int s = C.start[c]; s < e0; ++s) {
        const vec_t<T> qs = C.qB[s];
        for (int t = (di == 0) ? s + 1 : C.start[c1]; t < e1; ++t) {
            const vec_t<T> qt = C.qB[t];
            const T dx = (qs.x - qt.x) - sx;
            const T dy = (qs.y - qt.y) - sy;
            const T dz = (qs.z - qt.z) - sz;
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < C.rc2)
                ssa_pair(C, R, (uint32_t)rep, step, C.pB, C.eB, s, t, id_of(qs), id_of(qt), r2, dt, sqrt_dt);
        }
    }
}

__global__ void k_step_inc(long long* step) { *step += 1; }

// ---------------------------------------------------------------------------
// observables: per-chunk sums (a chunk lies inside one replica), then per
// replica sums of the chunks in order -- deterministic.
// terms: 0 K, 1 U, 2 Eint, 3-5 P, 6 sum C_v/eps, 7 |F|^2, 8 Laplacian U,
//        9 neg eps, 10 nonfinite
// ---------------------------------------------------------------------------
constexpr int NTERMS = 11;
constexpr int OBS_THREADS = 256;

template <class T>
__global__ void k_obs_chunks(Ctx<T> C, const int* __restrict__ chunk_rep, const int* __restrict__ chunk_begin,
                             const int* __restrict__ chunk_end, double* __restrict__ partial) {
    const int ch = blockIdx.x;
    const int rep = chunk_rep[ch];
    const RepInfo& R = C.reps[rep];
    double acc[NTERMS];
    for (int k = 0; k < NTERMS; ++k) acc[k] = 0.0;
    const double half_rc_a = 0.5 * (double)C.a * (double)C.rc;
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
            double u = 0.0, lap = 0.0;
            for_each_neighbour(C, C.qA, i, qi, C.cA[i], R,
                               [&](int, const vec_t<T>&, T, T, T, T r2, bool) {
                                   const double r = sqrt((double)r2);
                                   const double w = 1.0 - r / (double)C.rc;
                                   u += 0.5 * half_rc_a * w * w;   // each pair is seen twice
                                   if (r > 0.0) lap += (double)C.a / (double)C.rc - 2.0 * (double)C.a * w / r;
                               });
            acc[1] += u;
            acc[8] += lap;
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
