// dpde_device.cuh -- device-side building blocks of the DPDE step (sm_103a).
//
// Precision is a template parameter T: double for the FP64 mode, float for
// the mixed mode (internal energies stay double in both). Particle data are
// cell-sorted structures of arrays:
//   q   : (x, y, z, id bits)  -- the id rides in the 4th lane
//   p   : (px, py, pz, beta)  -- beta_i = C_v / eps_i, Eq. (DPDE_internalEOS)
//   F   : (Fx, Fy, Fz, -)
//   dp  : (dpx, dpy, dpz, -)  -- SER first-sweep sums delta p_i, Eq. (SER_p)
//   eps : double
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dpde {

// 32-byte aligned four-double vector (one 256-bit access per particle).
struct __align__(32) d4 {
    double x, y, z, w;
};

template <class T> struct V;
template <> struct V<double> { using t = d4; };
template <> struct V<float> { using t = float4; };
template <class T> using vec_t = typename V<T>::t;

__device__ __forceinline__ uint32_t id_of(const float4& q) { return __float_as_uint(q.w); }
__device__ __forceinline__ uint32_t id_of(const d4& q) {
    return (uint32_t)__double_as_longlong(q.w);
}
__device__ __forceinline__ void set_id(float4& q, uint32_t id) { q.w = __uint_as_float(id); }
__device__ __forceinline__ void set_id(d4& q, uint32_t id) {
    q.w = __longlong_as_double((long long)id);
}

// Per-replica constants (one independent periodic system each).
struct RepInfo {
    double L[3];     // box lengths
    double s[3];     // ncell_d / L_d, formed in double
    float Lf[3];     // float copies for the mixed mode
    float sf[3];
    int nc[3];       // cells per axis
    int k[3];        // cells per brick per axis
    int B[3];        // bricks (Hybrid domains) per axis
    int cell_off;    // first global cell index of the replica
    int ncells;
    int part_off;    // first particle slot of the replica
    int n;
    double cv;       // C_v
    float cvf;
    int odd_ring[3]; // brick periodic along axis (B == 1) with odd k
};

template <class T> __device__ __forceinline__ T box_len(const RepInfo& R, int d);
template <> __device__ __forceinline__ double box_len<double>(const RepInfo& R, int d) { return R.L[d]; }
template <> __device__ __forceinline__ float box_len<float>(const RepInfo& R, int d) { return R.Lf[d]; }
template <class T> __device__ __forceinline__ T cell_scale(const RepInfo& R, int d);
template <> __device__ __forceinline__ double cell_scale<double>(const RepInfo& R, int d) { return R.s[d]; }
template <> __device__ __forceinline__ float cell_scale<float>(const RepInfo& R, int d) { return R.sf[d]; }

// c_d(x) = min(ncell_d - 1, (int)(x * (ncell_d / L_d))) (x >= 0 after wrap).
template <class T>
__device__ __forceinline__ int cell_coord(T x, const RepInfo& R, int d) {
    int c = (int)(x * cell_scale<T>(R, d));
    c = c > R.nc[d] - 1 ? R.nc[d] - 1 : c;
    return c < 0 ? 0 : c;
}

__device__ __forceinline__ int cell_linear(const RepInfo& R, int cx, int cy, int cz) {
    return R.cell_off + (cz * R.nc[1] + cy) * R.nc[0] + cx;
}

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

// Status bits raised by the kernels (read and cleared by the host).
enum : unsigned int { ST_NEG_EPS = 1u, ST_NONFINITE = 2u };

}  // namespace dpde
