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

template <class T> struct Ctx {
    using vec = vec_t<T>;
    vec* qA; vec* pA; double* eA;
    vec* qB; vec* pB; double* eB;
    vec* F; vec* dp;
    int* key;        // global cell of each slot (A order)
    int* tmp;        // slots binned by cell, arbitrary order inside a cell
    int* count;      // per-cell counts (ncells), followed by fill (ncells)
    int* fill;
    int* start;      // ncells + 1 exclusive prefix of count
    const int* rep_of_slot;
    const int* rep_of_cell;
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
template <class T> __device__ __forceinline__ T wrap1(T x, T L) {
    if (x >= L) x -= L;
    else if (x < T(0)) x += L;
    return x;
}

template <class T> __device__ __forceinline__ T tsqrt(T x);
template <> __device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
template <class T> __device__ __forceinline__ T texpm1(T x);
template <> __device__ __forceinline__ float texpm1(float x) { return expm1f(x); }
template <> __device__ __forceinline__ double texpm1(double x) { return expm1(x); }

template <class T> __device__ __forceinline__ T beta_of(double eps, const RepInfo& R);
template <> __device__ __forceinline__ float beta_of<float>(double eps, const RepInfo& R) {
    return R.cvf / (float)eps;
}
template <> __device__ __forceinline__ double beta_of<double>(double eps, const RepInfo& R) {
    return R.cv / eps;
}

__device__ __forceinline__ void flag(unsigned int* st, unsigned int bits) { atomicOr(st, bits); }

template <class V> __device__ __forceinline__ bool finite3(const V& v) {
    return isfinite(v.x) && isfinite(v.y) && isfinite(v.z);
}

// Visits every neighbour j != i of slot i with |q_i - q_j| < r_cut (minimum
// image through the periodic shift of the wrapped neighbour cell), over the
// 27 cells around i's cell in (dz, dy, dx, slot) order. With cross_only, cells
// in the same brick as i's cell are skipped (Hybrid's SER over set A^c).
template <class T, class Body>
__device__ __forceinline__ void for_each_neighbour(const Ctx<T>& C, const vec_t<T>* __restrict__ q,
                                                   int i, const vec_t<T>& qi, const RepInfo& R,
                                                   bool cross_only, Body&& body) {
    const int cx = cell_coord<T>(qi.x, R, 0);
    const int cy = cell_coord<T>(qi.y, R, 1);
    const int cz = cell_coord<T>(qi.z, R, 2);
    const int bx = cx / R.k[0], by = cy / R.k[1], bz = cz / R.k[2];
    const T Lx = box_len<T>(R, 0), Ly = box_len<T>(R, 1), Lz = box_len<T>(R, 2);
    for (int dz = -1; dz <= 1; ++dz) {
        int z = cz + dz;
        T sz = T(0);
        if (z < 0) { z += R.nc[2]; sz = Lz; }
        else if (z >= R.nc[2]) { z -= R.nc[2]; sz = -Lz; }
        for (int dy = -1; dy <= 1; ++dy) {
            int y = cy + dy;
            T sy = T(0);
            if (y < 0) { y += R.nc[1]; sy = Ly; }
            else if (y >= R.nc[1]) { y -= R.nc[1]; sy = -Ly; }
            for (int dx = -1; dx <= 1; ++dx) {
                int x = cx + dx;
                T sx = T(0);
                if (x < 0) { x += R.nc[0]; sx = Lx; }
                else if (x >= R.nc[0]) { x -= R.nc[0]; sx = -Lx; }
                if (cross_only && x / R.k[0] == bx && y / R.k[1] == by && z / R.k[2] == bz)
                    continue;
                const int c = cell_linear(R, x, y, z);
                const int e = C.start[c + 1];
                for (int j = C.start[c]; j < e; ++j) {
                    if (j == i) continue;
                    const vec_t<T> qj = q[j];
                    const T ddx = (qi.x - qj.x) + sx;
                    const T ddy = (qi.y - qj.y) + sy;
                    const T ddz = (qi.z - qj.z) + sz;
                    const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                    if (r2 < C.rc2) body(j, qj, ddx, ddy, ddz, r2);
                }
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
    double xs[3];
    for (int d = 0; d < 3; ++d) {
        double x = q[3 * s + d];
        x -= R.L[d] * floor(x / R.L[d]);
        if (x >= R.L[d]) x -= R.L[d];
        xs[d] = x;
    }
    qv.x = (T)xs[0]; qv.y = (T)xs[1]; qv.z = (T)xs[2];
    // a value just below L can round up to L in float: fold it back to 0
    if (qv.x >= box_len<T>(R, 0)) qv.x = T(0);
    if (qv.y >= box_len<T>(R, 1)) qv.y = T(0);
    if (qv.z >= box_len<T>(R, 2)) qv.z = T(0);
    set_id(qv, (uint32_t)(s - R.part_off));
    pv.x = (T)p[3 * s]; pv.y = (T)p[3 * s + 1]; pv.z = (T)p[3 * s + 2];
    pv.w = beta_of<T>(e[s], R);
    C.qA[s] = qv;
    C.pA[s] = pv;
    C.eA[s] = e[s];
}

template <class T>
__global__ void k_get_state(Ctx<T> C, double* __restrict__ q, double* __restrict__ p,
                            double* __restrict__ e) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.N) return;
    const RepInfo& R = C.reps[C.rep_of_slot[s]];
    const vec_t<T> qv = C.qA[s];
    const vec_t<T> pv = C.pA[s];
    const long long g = (long long)R.part_off + id_of(qv);
    if (q) { q[3 * g] = (double)qv.x; q[3 * g + 1] = (double)qv.y; q[3 * g + 2] = (double)qv.z; }
    if (p) { p[3 * g] = (double)pv.x; p[3 * g + 1] = (double)pv.y; p[3 * g + 2] = (double)pv.z; }
    if (e) e[g] = C.eA[s];
}

// ---------------------------------------------------------------------------
// Verlet first half: p += dt/2 F; q += dt p / m; wrap. Then the cell key and
// the per-cell count of the sort.
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_kick_drift_key(Ctx<T> C, T half_dt, T dt, int kick) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.N) return;
    const RepInfo& R = C.reps[C.rep_of_slot[s]];
    vec_t<T> qv = C.qA[s];
    if (kick) {
        vec_t<T> pv = C.pA[s];
        const vec_t<T> f = C.F[s];
        pv.x += half_dt * f.x; pv.y += half_dt * f.y; pv.z += half_dt * f.z;
        const T c = dt * C.inv_m;
        qv.x = wrap1(qv.x + c * pv.x, box_len<T>(R, 0));
        qv.y = wrap1(qv.y + c * pv.y, box_len<T>(R, 1));
        qv.z = wrap1(qv.z + c * pv.z, box_len<T>(R, 2));
        C.pA[s] = pv;
        C.qA[s] = qv;
    }
    const int key = cell_linear(R, cell_coord<T>(qv.x, R, 0), cell_coord<T>(qv.y, R, 1),
                                cell_coord<T>(qv.z, R, 2));
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
    // warp inclusive scan, then scan of warp totals
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
    const double ev = C.eA[s];
    pv.w = beta_of<T>(ev, R);
    C.qB[dst] = qv;
    C.pB[dst] = pv;
    C.eB[dst] = ev;
}

// B -> A copy (after set_state and after the SSA-only scheme), refreshing beta
// and checking the state.
template <class T>
__global__ void k_copy_back(Ctx<T> C) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.N) return;
    const RepInfo& R = C.reps[C.rep_of_slot[s]];
    vec_t<T> pv = C.pB[s];
    const double ev = C.eB[s];
    pv.w = beta_of<T>(ev, R);
    C.qA[s] = C.qB[s];
    C.pA[s] = pv;
    C.eA[s] = ev;
    if (!(ev > 0.0)) flag(C.status, ST_NEG_EPS);
    if (!finite3(pv) || !isfinite(ev)) flag(C.status, ST_NONFINITE);
}

template <class T>
__global__ void k_refresh_beta(Ctx<T> C) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.N) return;
    C.pB[s].w = beta_of<T>(C.eB[s], C.reps[C.rep_of_slot[s]]);
}

// ---------------------------------------------------------------------------
// conservative forces F(q) on B (soft repulsion a (1 - r/r_cut) r_hat), then
// the second Verlet half-kick p += dt/2 F when kick != 0
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_force(Ctx<T> C, T half_dt, int kick) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.N) return;
    const RepInfo& R = C.reps[C.rep_of_slot[i]];
    const vec_t<T> qi = C.qB[i];
    T fx = 0, fy = 0, fz = 0;
    for_each_neighbour(C, C.qB, i, qi, R, false,
                       [&](int, const vec_t<T>&, T dx, T dy, T dz, T r2) {
                           if (r2 > T(0)) {
                               const T r = tsqrt(r2);
                               const T f = C.a * (T(1) - r * C.inv_rc) / r;
                               fx += f * dx; fy += f * dy; fz += f * dz;
                           }
                       });
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
// SER (Sec. III.B.1). delta p_ij = -gamma_ij chi v_ij dt + sigma sqrt(chi)
// G_ij sqrt(dt), gamma_ij = sigma^2/4 (beta_i + beta_j) (Eq. DPDE_fd).
// ---------------------------------------------------------------------------
template <class T>
struct PairFD {
    T A;   // -gamma chi dt
    T Bn;  // sigma sqrt(chi) sqrt(dt)
};

template <class T>
__device__ __forceinline__ PairFD<T> pair_coeffs(const Ctx<T>& C, T r2, T beta_i, T beta_j, T dt,
                                                 T sqrt_dt) {
    const T r = tsqrt(r2);
    const T w = T(1) - r * C.inv_rc;
    const T gam = C.sig2_4 * (beta_i + beta_j);
    return {-gam * (w * w) * dt, C.sigma * w * sqrt_dt};
}

// first sweep: delta p_i = sum_j delta p_ij (Eq. SER_p)
template <class T>
__global__ void k_ser_sweep1(Ctx<T> C, T dt, T sqrt_dt, int cross_only) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.N) return;
    const int rep = C.rep_of_slot[i];
    const RepInfo& R = C.reps[rep];
    const vec_t<T> qi = C.qB[i];
    const vec_t<T> pi = C.pB[i];
    const uint32_t idi = id_of(qi);
    const uint32_t step = (uint32_t)*C.step;
    T ax = 0, ay = 0, az = 0;
    for_each_neighbour(C, C.qB, i, qi, R, cross_only != 0,
                       [&](int j, const vec_t<T>& qj, T, T, T, T r2) {
                           const vec_t<T> pj = C.pB[j];
                           const PairFD<T> k = pair_coeffs(C, r2, pi.w, pj.w, dt, sqrt_dt);
                           const T3<T> G = pair_gauss<T>(C.seed, step, (uint32_t)rep, idi, id_of(qj));
                           const T vx = (pi.x - pj.x) * C.inv_m;
                           const T vy = (pi.y - pj.y) * C.inv_m;
                           const T vz = (pi.z - pj.z) * C.inv_m;
                           ax += k.A * vx + k.Bn * G.x;
                           ay += k.A * vy + k.Bn * G.y;
                           az += k.A * vz + k.Bn * G.z;
                       });
    vec_t<T> out;
    out.x = ax; out.y = ay; out.z = az; out.w = T(0);
    C.dp[i] = out;
}

// second sweep, Eq. (SER_eint_discretization), in the equivalent form
//   Delta eps_i = -Delta K_i + 1/2 sum_j T_ij,
//   T_ij = delta p_ij . (v_i + v_j + (delta p_i + delta p_j) / (2m)),
// where Delta K_i is the kinetic-energy change of the stored momenta,
// evaluated in double. T_ij = -T_ji bit for bit, so the FD part conserves the
// double-evaluated energy up to the rounding of the per-particle sums.
// Writes p + delta p, eps + Delta eps and q into set A.
template <class T>
__global__ void k_ser_sweep2(Ctx<T> C, T dt, T sqrt_dt, int cross_only) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.N) return;
    const int rep = C.rep_of_slot[i];
    const RepInfo& R = C.reps[rep];
    const vec_t<T> qi = C.qB[i];
    const vec_t<T> pi = C.pB[i];
    const vec_t<T> dpi = C.dp[i];
    const uint32_t idi = id_of(qi);
    const uint32_t step = (uint32_t)*C.step;
    const T hm = T(0.5) * C.inv_m;
    const T vix = pi.x * C.inv_m, viy = pi.y * C.inv_m, viz = pi.z * C.inv_m;
    T tsum = 0;
    for_each_neighbour(C, C.qB, i, qi, R, cross_only != 0,
                       [&](int j, const vec_t<T>& qj, T, T, T, T r2) {
                           const vec_t<T> pj = C.pB[j];
                           const vec_t<T> dpj = C.dp[j];
                           const PairFD<T> k = pair_coeffs(C, r2, pi.w, pj.w, dt, sqrt_dt);
                           const T3<T> G = pair_gauss<T>(C.seed, step, (uint32_t)rep, idi, id_of(qj));
                           const T vjx = pj.x * C.inv_m, vjy = pj.y * C.inv_m, vjz = pj.z * C.inv_m;
                           const T dx = k.A * (vix - vjx) + k.Bn * G.x;
                           const T dy = k.A * (viy - vjy) + k.Bn * G.y;
                           const T dz = k.A * (viz - vjz) + k.Bn * G.z;
                           tsum += dx * ((vix + vjx) + (dpi.x + dpj.x) * hm) +
                                   dy * ((viy + vjy) + (dpi.y + dpj.y) * hm) +
                                   dz * ((viz + vjz) + (dpi.z + dpj.z) * hm);
                       });
    vec_t<T> pn = pi;
    pn.x = pi.x + dpi.x; pn.y = pi.y + dpi.y; pn.z = pi.z + dpi.z;
    const double dK = (((double)pn.x - (double)pi.x) * ((double)pn.x + (double)pi.x) +
                       ((double)pn.y - (double)pi.y) * ((double)pn.y + (double)pi.y) +
                       ((double)pn.z - (double)pi.z) * ((double)pn.z + (double)pi.z)) *
                      (0.5 / (double)C.m);
    const double en = C.eB[i] - dK + 0.5 * (double)tsum;
    pn.w = beta_of<T>(en, R);
    C.qA[i] = qi;
    C.pA[i] = pn;
    C.eA[i] = en;
    if (!(en > 0.0)) flag(C.status, ST_NEG_EPS);
    if (!finite3(pn) || !isfinite(en)) flag(C.status, ST_NONFINITE);
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
    const vec_t<T> qi = C.qB[i];
    const vec_t<T> pi = C.pB[i];
    const uint32_t idi = id_of(qi);
    const uint32_t step = (uint32_t)*C.step;
    const T d_sig2_m = T(3) * C.sigma * C.sigma * C.inv_m;
    T ax = 0, ay = 0, az = 0, de = 0;
    for_each_neighbour(C, C.qB, i, qi, R, false,
                       [&](int j, const vec_t<T>& qj, T, T, T, T r2) {
                           const vec_t<T> pj = C.pB[j];
                           const T r = tsqrt(r2);
                           const T w = T(1) - r * C.inv_rc;
                           const T chi = w * w;
                           const T gam = C.sig2_4 * (pi.w + pj.w);
                           const T3<T> G = pair_gauss<T>(C.seed, step, (uint32_t)rep, idi, id_of(qj));
                           const T vx = (pi.x - pj.x) * C.inv_m;
                           const T vy = (pi.y - pj.y) * C.inv_m;
                           const T vz = (pi.z - pj.z) * C.inv_m;
                           const T A = -gam * chi * dt, Bn = C.sigma * w * sqrt_dt;
                           ax += A * vx + Bn * G.x;
                           ay += A * vy + Bn * G.y;
                           az += A * vz + Bn * G.z;
                           de += T(0.5) * (gam * (vx * vx + vy * vy + vz * vz) - d_sig2_m) * chi * dt -
                                 T(0.5) * Bn * (vx * G.x + vy * G.y + vz * G.z);
                       });
    vec_t<T> pn = pi;
    pn.x = pi.x + ax; pn.y = pi.y + ay; pn.z = pi.z + az;
    const double en = C.eB[i] + (double)de;
    pn.w = beta_of<T>(en, R);
    C.qA[i] = qi;
    C.pA[i] = pn;
    C.eA[i] = en;
    if (!(en > 0.0)) flag(C.status, ST_NEG_EPS);
    if (!finite3(pn) || !isfinite(en)) flag(C.status, ST_NONFINITE);
}

// ---------------------------------------------------------------------------
// SSA rounds (Eq. SSA_ij) -- one launch per (direction, colour); the cell
// pairs of a round touch disjoint particles, so they run in parallel and
// update B in place. Sequence definition: see the library header.
// ---------------------------------------------------------------------------
__constant__ int c_dirs[14][3] = {{0, 0, 0},   {1, 0, 0},  {-1, 1, 0}, {0, 1, 0},  {1, 1, 0},
                                  {-1, -1, 1}, {0, -1, 1}, {1, -1, 1}, {-1, 0, 1}, {0, 0, 1},
                                  {1, 0, 1},   {-1, 1, 1}, {0, 1, 1},  {1, 1, 1}};

template <class T>
__device__ __forceinline__ void ssa_pair(const Ctx<T>& C, const RepInfo& R, int rep, uint32_t step,
                                         int s, int t, T r2, T dt, T sqrt_dt) {
    vec_t<T> ps = C.pB[s], pt = C.pB[t];
    double es = C.eB[s], et = C.eB[t];
    const T r = tsqrt(r2);
    const T w = T(1) - r * C.inv_rc;
    const T chi = w * w;
    const T gam = C.sig2_4 * (beta_of<T>(es, R) + beta_of<T>(et, R));
    const T a = T(2) * gam * chi * dt * C.inv_m;
    const T amp = (gam != T(0)) ? C.sigma * tsqrt(C.m * (-texpm1(T(-2) * a)) / gam)
                                : T(2) * C.sigma * w * sqrt_dt;
    const T em1 = texpm1(-a);
    const T3<T> G = pair_gauss<T>(C.seed, step, (uint32_t)rep, id_of(C.qB[s]), id_of(C.qB[t]));
    const T Dx = T(0.5) * (em1 * (ps.x - pt.x) + amp * G.x);
    const T Dy = T(0.5) * (em1 * (ps.y - pt.y) + amp * G.y);
    const T Dz = T(0.5) * (em1 * (ps.z - pt.z) + amp * G.z);
    vec_t<T> sn = ps, tn = pt;
    sn.x = ps.x + Dx; sn.y = ps.y + Dy; sn.z = ps.z + Dz;
    tn.x = pt.x - Dx; tn.y = pt.y - Dy; tn.z = pt.z - Dz;
    const double dK = (((double)sn.x - (double)ps.x) * ((double)sn.x + (double)ps.x) +
                       ((double)sn.y - (double)ps.y) * ((double)sn.y + (double)ps.y) +
                       ((double)sn.z - (double)ps.z) * ((double)sn.z + (double)ps.z) +
                       ((double)tn.x - (double)pt.x) * ((double)tn.x + (double)pt.x) +
                       ((double)tn.y - (double)pt.y) * ((double)tn.y + (double)pt.y) +
                       ((double)tn.z - (double)pt.z) * ((double)tn.z + (double)pt.z)) *
                      (0.5 / (double)C.m);
    C.pB[s] = sn;
    C.pB[t] = tn;
    C.eB[s] = es - 0.5 * dK;
    C.eB[t] = et - 0.5 * dK;
}

template <class T>
__global__ void k_ssa_round(Ctx<T> C, int di, int col, int whole_box, T dt, T sqrt_dt) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C.ncells) return;
    const int rep = C.rep_of_cell[c];
    const RepInfo& R = C.reps[rep];
    const int lc = c - R.cell_off;
    const int cc[3] = {lc % R.nc[0], (lc / R.nc[0]) % R.nc[1], lc / (R.nc[0] * R.nc[1])};
    int B[3], k[3];
    for (int d = 0; d < 3; ++d) {
        B[d] = whole_box ? 1 : R.B[d];
        k[d] = whole_box ? R.nc[d] : R.k[d];
    }
    const int* del = c_dirs[di];
    const int lead = del[2] != 0 ? 2 : (del[1] != 0 ? 1 : 0);
    if (di > 0) {
        const int l = cc[lead] % k[lead];
        const bool odd = (B[lead] == 1) && (k[lead] & 1);
        const int my = (odd && l == k[lead] - 1) ? 2 : (l & 1);
        if (my != col) return;
    }
    int nb[3];
    T sh[3];
    for (int d = 0; d < 3; ++d) {
        const int l = cc[d] % k[d];
        int ln = l + del[d];
        sh[d] = T(0);
        if (B[d] == 1) {
            if (ln < 0) { ln += k[d]; sh[d] = box_len<T>(R, d); }
            else if (ln >= k[d]) { ln -= k[d]; sh[d] = -box_len<T>(R, d); }
        } else if (ln < 0 || ln >= k[d]) {
            return;
        }
        nb[d] = (cc[d] / k[d]) * k[d] + ln;
    }
    const int c1 = cell_linear(R, nb[0], nb[1], nb[2]);
    const uint32_t step = (uint32_t)*C.step;
    const int e0 = C.start[c + 1], e1 = C.start[c1 + 1];
    for (int s = C.start[c]; s < e0; ++s) {
        const vec_t<T> qs = C.qB[s];
        for (int t = (di == 0) ? s + 1 : C.start[c1]; t < e1; ++t) {
            const vec_t<T> qt = C.qB[t];
            const T dx = (qs.x - qt.x) + sh[0];
            const T dy = (qs.y - qt.y) + sh[1];
            const T dz = (qs.z - qt.z) + sh[2];
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < C.rc2) ssa_pair(C, R, rep, step, s, t, r2, dt, sqrt_dt);
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
        const double e = C.eA[i];
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
            for_each_neighbour(C, C.qA, i, qi, R, false, [&](int, const vec_t<T>&, T, T, T, T r2) {
                const double r = sqrt((double)r2);
                const double w = 1.0 - r / (double)C.rc;
                u += 0.5 * half_rc_a * w * w;   // half of v(r): each pair is seen twice
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
