// dpde_device.cuh -- device-side building blocks of the DPDE step (sm_103a).
//
// Precision is a template parameter T of positions, momenta, forces and pair
// arithmetic: double (FP64 mode) or float (mixed mode). Internal energies use
// the type E: double in FP64 mode, a compensated float pair (hi + lo, about
// 48 significant bits) in the mixed mode, so that the small per-pair energy
// reinjections are not lost against eps ~ C_v T.
//
// Particle data are cell-sorted structures of arrays (slot order):
//   q   : (ox, oy, oz, id bits) -- offset of the particle inside its cell,
//                                  o in [0, l) with l = L / ncell per axis
//   cc  : packed cell coordinates cx | cy << 10 | cz << 20
//   p   : (px, py, pz, beta)    -- beta_i = C_v / eps_i, Eq. (DPDE_internalEOS)
//   eps : E
// Cell-relative offsets keep float positions at ~1e-7 absolute resolution
// whatever the box size; the distance between particles of cells c and
// c + d is (o_i - o_j) - d * l, which also gives the periodic image.
#pragma once

#include <cmath>

#include <cstdint>
#include <cuda_runtime.h>

namespace dpde {

// 32-byte aligned four-double vector (one 256-bit access per particle).
struct __align__(32) d4 {
    double x, y, z, w;
};

// Compensated float pair: value = hi + lo with |lo| <= ulp(hi)/2.
struct __align__(8) ff {
    float hi, lo;
};

template <class T> struct V;
template <> struct V<double> { using t = d4; using e = double; };
template <> struct V<float> { using t = float4; using e = ff; };
template <class T> using vec_t = typename V<T>::t;
template <class T> using eps_t = typename V<T>::e;

__device__ __forceinline__ uint32_t id_of(const float4& q) { return __float_as_uint(q.w); }
__device__ __forceinline__ uint32_t id_of(const d4& q) {
    return (uint32_t)__double_as_longlong(q.w);
}
__device__ __forceinline__ void set_id(float4& q, uint32_t id) { q.w = __uint_as_float(id); }
__device__ __forceinline__ void set_id(d4& q, uint32_t id) {
    q.w = __longlong_as_double((long long)id);
}

// ---------------------------------------------------------------------------
// compensated float arithmetic (Knuth's two-sum; Dekker's normalisation)
// ---------------------------------------------------------------------------
__device__ __forceinline__ ff ff_add(ff a, float b) {
    const float s = __fadd_rn(a.hi, b);
    const float bb = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    const float lo = __fadd_rn(a.lo, err);
    const float hi = __fadd_rn(s, lo);
    return {hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}
// Knuth's two-sum: a + b = s + err exactly
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}
// compensated pair + compensated pair (normalised)
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    float e;
    const float s = two_sum(a.hi, b.hi, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, e);
    return {hi, __fsub_rn(e, __fsub_rn(hi, s))};
}
// (p1 - p0)(p1 + p0) of two floats as hi + lo, to a few units of 2^-46 of
// its size: both factors by two-sum, their leading product by the FMA
// two-product (its rounding error exactly), the cross terms in float.
__device__ __forceinline__ float diff_of_squares(float p1, float p0, float& lo) {
    float ea, eb;
    const float a = two_sum(p1, -p0, ea);
    const float b = two_sum(p1, p0, eb);
    const float h = __fmul_rn(a, b);
    lo = __fadd_rn(__fmaf_rn(a, b, -h), __fadd_rn(__fmul_rn(a, eb), __fmul_rn(ea, b)));
    return h;
}
__device__ __forceinline__ double eps_value(double e) { return e; }
__device__ __forceinline__ double eps_value(ff e) { return (double)e.hi + (double)e.lo; }
__device__ __forceinline__ void eps_from(double v, double& e) { e = v; }
__device__ __forceinline__ void eps_from(double v, ff& e) {
    e.hi = (float)v;
    e.lo = (float)(v - (double)e.hi);
}
__device__ __forceinline__ double eps_add(double e, double d) { return e + d; }
__device__ __forceinline__ ff eps_add(ff e, float d) { return ff_add(e, d); }

// Per-replica constants (one independent periodic system each).
struct RepInfo {
    double L[3];     // box lengths
    double ell[3];   // cell size L_d / ncell_d
    double s[3];     // ncell_d / L_d
    float ellf[3];
    int nc[3];       // cells per axis
    int k[3];        // cells per brick per axis
    int B[3];        // bricks (Hybrid domains) per axis
    int cell_off;    // first global cell index of the replica
    int ncells;
    int part_off;    // first particle slot of the replica
    int n;
    int brick_off;   // first global brick index of the replica
    int tab_off;     // offset of the replica's cell tables
    double cv;       // C_v
    float cvf;
    int walls;       // 1: specular walls along z (not periodic along z)
    double wall_u;   // velocity of the upper wall along z (walls = 1)
};

// Position of the upper wall of a walled replica for the current step's
// drift, as a cell index and an offset in it: z_w = c ell_z + o.
struct WallPos {
    double o;
    int c;
    int pad;
};

// Cell tables of a replica, at tab_off: lin_x[nc0] | lin_y[nc1] | lin_z[nc2]
// | brick_x[nc0] | brick_y[nc1] | brick_z[nc2]. The brick-major linear cell
// index is cell_off + lin_x[cx] + lin_y[cy] + lin_z[cz]; brick_d[c] = c / k_d.
__device__ __forceinline__ int cell_index(const int* __restrict__ tab, const RepInfo& R, int cx,
                                          int cy, int cz) {
    const int* t = tab + R.tab_off;
    return R.cell_off + __ldg(t + cx) + __ldg(t + R.nc[0] + cy) + __ldg(t + R.nc[0] + R.nc[1] + cz);
}
__device__ __forceinline__ const int* brick_tab(const int* __restrict__ tab, const RepInfo& R) {
    return tab + R.tab_off + R.nc[0] + R.nc[1] + R.nc[2];
}

__device__ __forceinline__ int pack_cell(int cx, int cy, int cz) { return cx | (cy << 10) | (cz << 20); }
__device__ __forceinline__ int cell_x(int c) { return c & 1023; }
__device__ __forceinline__ int cell_y(int c) { return (c >> 10) & 1023; }
__device__ __forceinline__ int cell_z(int c) { return (c >> 20) & 1023; }

template <class T> __device__ __forceinline__ T cell_len(const RepInfo& R, int d);
template <> __device__ __forceinline__ double cell_len<double>(const RepInfo& R, int d) { return R.ell[d]; }
template <> __device__ __forceinline__ float cell_len<float>(const RepInfo& R, int d) { return R.ellf[d]; }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round
// multiplies counter words 0 and 2 by the two round constants, keeps the full
// 64-bit products, and xors the high halves with words 1 / 3 and the key;
// the key is advanced by the two Weyl constants before every later round.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

template <class T> struct T3 { T x, y, z; };

// Box-Muller on 24-bit uniforms u in (0, 1] and t in [0, 1) (exact in float):
// G = (R1 cos 2 pi t1, R1 sin 2 pi t1, R2 cos 2 pi t2), R = sqrt(-2 ln u).
__device__ __forceinline__ T3<float> gauss3(uint4 x, float) {
    const float u1 = (float)((x.x >> 8) + 1u) * 0x1p-24f;
    const float t1 = (float)(x.y >> 8) * 0x1p-24f;
    const float u2 = (float)((x.z >> 8) + 1u) * 0x1p-24f;
    const float t2 = (float)(x.w >> 8) * 0x1p-24f;
    const float R1 = sqrtf(-2.0f * logf(u1));
    const float R2 = sqrtf(-2.0f * logf(u2));
    float s1, c1;
    sincospif(2.0f * t1, &s1, &c1);
    const float c2 = cospif(2.0f * t2);
    return {R1 * c1, R1 * s1, R2 * c2};
}
__device__ __forceinline__ T3<double> gauss3(uint4 x, double) {
    const double u1 = (double)((x.x >> 8) + 1u) * 0x1p-24;
    const double t1 = (double)(x.y >> 8) * 0x1p-24;
    const double u2 = (double)((x.z >> 8) + 1u) * 0x1p-24;
    const double t2 = (double)(x.w >> 8) * 0x1p-24;
    const double R1 = sqrt(-2.0 * log(u1));
    const double R2 = sqrt(-2.0 * log(u2));
    double s1, c1;
    sincospi(2.0 * t1, &s1, &c1);
    const double c2 = cospi(2.0 * t2);
    return {R1 * c1, R1 * s1, R2 * c2};
}

// G_ij for particle i (id_i) and neighbour j (id_j): drawn for the ordered
// pair (min id, max id) and negated when id_i > id_j, so G_ji = -G_ij.
template <class T>
__device__ __forceinline__ T3<T> pair_gauss(uint2 key, uint32_t step, uint32_t rep, uint32_t id_i,
                                            uint32_t id_j) {
    const bool lo = id_i < id_j;
    const uint4 x = philox4x32_10(make_uint4(lo ? id_i : id_j, lo ? id_j : id_i, step, rep), key);
    T3<T> g = gauss3(x, T(0));
    if (!lo) {
        g.x = -g.x;
        g.y = -g.y;
        g.z = -g.z;
    }
    return g;
}

// ---------------------------------------------------------------------------
// Pair potential: the soft repulsion v = (a r_c/2)(1 - r/r_c)^2, or the
// shifted, splined, truncated Lennard-Jones potential of Eq. (Ep),
// v = 4 eps((r_LJ/r)^12 - (r_LJ/r)^6) - eps_sh - f_sp (r - r_c) with eps_sh =
// v_LJ(r_c), f_sp = v_LJ'(r_c) so that v(r_c) = v'(r_c) = 0.
// ---------------------------------------------------------------------------
template <class T> struct PotT {
    int kind;                       // DPDE_POT_SOFT or DPDE_POT_LJ
    T a, rc, inv_rc, half_arc;      // soft: a, r_c, 1/r_c, a r_c / 2
    T lj4e, ljr2, ljesh, ljfsp;     // LJ: 4 eps, r_LJ^2, eps_sh, f_sp
};

// For 0 < r2 < r_c^2 and ir = 1/sqrt(r2): v(r), fr = -v'(r)/r (so that the
// force on i is fr (q_i - q_j)) and lap = v''(r) + 2 v'(r)/r.
template <class T>
__device__ __forceinline__ void pair_pot(const PotT<T>& P, T r2, T ir, T& v, T& fr, T& lap) {
    const T r = r2 * ir;
    if (P.kind == 1) {
        const T ir2 = ir * ir;
        const T s2 = P.ljr2 * ir2, s6 = s2 * s2 * s2, s12 = s6 * s6;
        const T dv = P.lj4e * (T(6) * s6 - T(12) * s12) * ir - P.ljfsp;
        v = P.lj4e * (s12 - s6) - P.ljesh - P.ljfsp * (r - P.rc);
        fr = -dv * ir;
        lap = P.lj4e * (T(156) * s12 - T(42) * s6) * ir2 + T(2) * dv * ir;
    } else {
        const T w = T(1) - r * P.inv_rc;
        v = P.half_arc * w * w;
        fr = P.a * w * ir;
        lap = P.a * P.inv_rc - T(2) * P.a * w * ir;
    }
}

// Constants of the pair potential from the parameters (host side, double).
inline PotT<double> make_pot(int kind, double a, double rc, double lj_eps, double lj_r) {
    PotT<double> P{};
    P.kind = kind;
    P.a = a;
    P.rc = rc;
    P.inv_rc = 1.0 / rc;
    P.half_arc = 0.5 * a * rc;
    if (kind == 1) {
        const double s6 = std::pow(lj_r / rc, 6.0), s12 = s6 * s6;
        P.lj4e = 4.0 * lj_eps;
        P.ljr2 = lj_r * lj_r;
        P.ljesh = 4.0 * lj_eps * (s12 - s6);                  // v_LJ(r_c)
        P.ljfsp = 4.0 * lj_eps * (6.0 * s6 - 12.0 * s12) / rc;  // v_LJ'(r_c)
    }
    return P;
}

template <class T> inline PotT<T> cast_pot(const PotT<double>& P) {
    return PotT<T>{P.kind, (T)P.a, (T)P.rc, (T)P.inv_rc, (T)P.half_arc, (T)P.lj4e, (T)P.ljr2, (T)P.ljesh, (T)P.ljfsp};
}

// v at r = 0: the soft potential's maximum; no LJ term
template <class T>
__device__ __forceinline__ T pair_pot_at_zero(const PotT<T>& P) { return P.kind == 1 ? T(0) : P.half_arc; }

// Status bits raised by the kernels (read and cleared by the host).
enum : unsigned int {
    ST_NEG_EPS = 1u, ST_NONFINITE = 2u, ST_CAPACITY = 4u, ST_DOMAIN = 8u, ST_WALL = 16u, ST_TIMEOUT = 32u
};

}  // namespace dpde
