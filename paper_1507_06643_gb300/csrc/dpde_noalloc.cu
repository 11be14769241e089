// dpde_noalloc.cu -- observables of one system without any device allocation.
//
// For callers that cannot call cudaMalloc: plug-ins living inside a host
// framework that owns all device memory through its own pool (a side
// allocation would fail, or fragment and outgrow the pool's budget), and
// processes under a hard device-memory cap or with a no-allocation rule after
// start-up. The caller passes the state (device arrays) and receives the
// observables; all working memory comes from one file-scope device array of
// fixed size (SCRATCH_BYTES below, held by every GPU that loads the library
// until the process exits). Every call shares that array: calls that overlap
// on the GPU (different streams or threads using the same device) race and
// must be serialised by the caller. The first call on a device looks up the
// array's device address with cudaGetSymbolAddress (set-up); that first call
// should come before any stream capture begins. Each call waits for its
// stream before returning, to hand back the results.
#include "dpde.h"
#include "dpde_device.cuh"

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

namespace {

constexpr int NA_MAX_N = DPDE_NOALLOC_MAX_N;
constexpr int NA_MAX_CELLS = DPDE_NOALLOC_MAX_CELLS;
constexpr int NA_BLOCKS = 256;        // partial-sum blocks of the reduction
constexpr int NA_THREADS = 256;
constexpr int NA_TERMS = 11;

// scratch layout (bytes, 256-aligned sections)
constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_COUNT = 0;
constexpr size_t OFF_START = OFF_COUNT + al(sizeof(int) * NA_MAX_CELLS);
constexpr size_t OFF_FILL = OFF_START + al(sizeof(int) * (NA_MAX_CELLS + 1));
constexpr size_t OFF_PERM = OFF_FILL + al(sizeof(int) * NA_MAX_CELLS);
constexpr size_t OFF_PART = OFF_PERM + al(sizeof(int) * NA_MAX_N);
constexpr size_t OFF_OUT = OFF_PART + al(sizeof(double) * NA_BLOCKS * NA_TERMS);
constexpr size_t SCRATCH_BYTES = OFF_OUT + al(sizeof(double) * NA_TERMS);
static_assert(SCRATCH_BYTES == DPDE_NOALLOC_SCRATCH_BYTES, "scratch size in dpde.h is stale");

}  // namespace

// Device-side scratch of the no-allocation entry point. In host code this
// name is only a host-side stand-in: kernels get the device address obtained
// with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

namespace {

thread_local std::string g_na_error;
std::mutex g_na_mutex;
constexpr int NA_MAX_DEVICES = 64;
unsigned char* g_na_ptr[NA_MAX_DEVICES] = {};

struct NaGeom {
    double L[3], s[3];
    int nc[3];
    double rc, rc2, a, mass, cv;
    int n;
    int walls;   // 1: walls along z (no periodic image along z)
    dpde::PotT<double> pot;
};

// Cell coordinate along axis d: periodic axes wrap x into [0, L); the z axis
// of a walled replica does not wrap (a particle on the upper wall face, z =
// L_z, belongs to the top cell layer, one at z = 0 to the bottom one).
__device__ __forceinline__ int na_cell(const NaGeom& G, const double* q, int i, int d) {
    double x = q[3 * i + d];
    if (!(d == 2 && G.walls)) x -= G.L[d] * floor(x / G.L[d]);
    const double f = floor(x * G.s[d]);
    if (!(f >= 0.0)) return 0;
    return f >= (double)(G.nc[d] - 1) ? G.nc[d] - 1 : (int)f;
}

__device__ __forceinline__ int na_lin(const NaGeom& G, int cx, int cy, int cz) {
    return (cz * G.nc[1] + cy) * G.nc[0] + cx;
}

__global__ void k_na_count(NaGeom G, const double* __restrict__ q, int* __restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G.n) return;
    atomicAdd(&count[na_lin(G, na_cell(G, q, i, 0), na_cell(G, q, i, 1), na_cell(G, q, i, 2))], 1);
}

// single-block exclusive scan of the cell counts
__global__ void k_na_scan(const int* __restrict__ count, int* __restrict__ start, int ncells) {
    __shared__ int sh[NA_THREADS];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < ncells; b0 += NA_THREADS) {
        const int c = b0 + threadIdx.x;
        const int v = c < ncells ? count[c] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < NA_THREADS; o <<= 1) {
            const int y = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += y;
            __syncthreads();
        }
        if (c < ncells) start[c] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == NA_THREADS - 1) carry += sh[NA_THREADS - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) start[ncells] = carry;
}

__global__ void k_na_scatter(NaGeom G, const double* __restrict__ q, const int* __restrict__ start,
                             int* __restrict__ fill, int* __restrict__ perm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G.n) return;
    const int c = na_lin(G, na_cell(G, q, i, 0), na_cell(G, q, i, 1), na_cell(G, q, i, 2));
    perm[start[c] + atomicAdd(&fill[c], 1)] = i;
}

// per-particle terms (as dpde_observables: K, U, Eint, P, sum C_v/eps,
// |F|^2, Laplacian U, eps <= 0 count, non-finite count), one partial sum per
// block over a grid-stride range
__global__ void k_na_terms(NaGeom G, const double* __restrict__ q, const double* __restrict__ p,
                           const double* __restrict__ e, const int* __restrict__ start,
                           const int* __restrict__ perm, double* __restrict__ partial) {
    double acc[NA_TERMS];
    for (int k = 0; k < NA_TERMS; ++k) acc[k] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.n; i += gridDim.x * blockDim.x) {
        const double px = p[3 * i], py = p[3 * i + 1], pz = p[3 * i + 2], ei = e[i];
        double xi[3];
        bool fin = isfinite(px) && isfinite(py) && isfinite(pz) && isfinite(ei);
        for (int d = 0; d < 3; ++d) {
            xi[d] = q[3 * i + d];
            fin = fin && isfinite(xi[d]);
        }
        acc[0] += (px * px + py * py + pz * pz) / (2.0 * G.mass);
        acc[2] += ei;
        acc[3] += px; acc[4] += py; acc[5] += pz;
        acc[6] += G.cv / ei;
        acc[9] += ei <= 0.0 ? 1.0 : 0.0;
        acc[10] += fin ? 0.0 : 1.0;
        if (!fin) continue;
        const int cx = na_cell(G, q, i, 0), cy = na_cell(G, q, i, 1), cz = na_cell(G, q, i, 2);
        double fx = 0, fy = 0, fz = 0, u = 0, lap = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (G.walls && (cz + dz < 0 || cz + dz >= G.nc[2])) continue;
                    const int x = (cx + dx + G.nc[0]) % G.nc[0];
                    const int y = (cy + dy + G.nc[1]) % G.nc[1];
                    const int z = (cz + dz + G.nc[2]) % G.nc[2];
                    const int c = na_lin(G, x, y, z);
                    for (int k = start[c]; k < start[c + 1]; ++k) {
                        const int j = perm[k];
                        if (j == i) continue;
                        double d[3], r2 = 0.0;
                        for (int a = 0; a < 3; ++a) {
                            double v = xi[a] - q[3 * j + a];
                            if (!(a == 2 && G.walls)) v -= G.L[a] * rint(v / G.L[a]);
                            d[a] = v;
                            r2 += v * v;
                        }
                        if (!(r2 < G.rc2)) continue;   // also drops a NaN separation
                        if (r2 > 0.0) {
                            double v, fr, lp;
                            dpde::pair_pot(G.pot, r2, 1.0 / sqrt(r2), v, fr, lp);
                            u += 0.5 * v;   // each pair is seen twice
                            fx += fr * d[0]; fy += fr * d[1]; fz += fr * d[2];
                            lap += lp;
                        } else {
                            u += 0.5 * dpde::pair_pot_at_zero(G.pot);
                        }
                    }
                }
        acc[1] += u;
        acc[7] += fx * fx + fy * fy + fz * fz;
        acc[8] += lap;
    }
    __shared__ double sh[NA_TERMS][NA_THREADS];
    for (int k = 0; k < NA_TERMS; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < NA_TERMS; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < NA_TERMS) partial[blockIdx.x * NA_TERMS + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_na_final(const double* __restrict__ partial, double* __restrict__ out) {
    if (threadIdx.x >= NA_TERMS) return;
    double s = 0.0;
    for (int b = 0; b < NA_BLOCKS; ++b) s += partial[b * NA_TERMS + threadIdx.x];
    out[threadIdx.x] = s;
}

int na_fail(int code, const std::string& msg) {
    g_na_error = msg;
    return code;
}

// A state pointer must be device (or managed) memory reachable from the
// current device: a host pointer given to the kernels would fault, or on a
// system where the GPU can read host memory silently read the wrong data.
int na_check_device_ptr(const void* ptr, int dev, const char* name) {
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();   // the failed query is not sticky: clear it
        return na_fail(DPDE_ERR_ARG, std::string(name) + " is not a CUDA device pointer (" +
                                         cudaGetErrorString(e) + ")");
    }
    if (a.type == cudaMemoryTypeManaged) return DPDE_OK;
    if (a.type != cudaMemoryTypeDevice)
        return na_fail(DPDE_ERR_ARG, std::string(name) + " must point to device memory (got a host pointer)");
    if (a.device != dev)
        return na_fail(DPDE_ERR_ARG, std::string(name) + " lives on device " + std::to_string(a.device) +
                                         ", not on the current device " + std::to_string(dev));
    return DPDE_OK;
}

}  // namespace

extern "C" {

int dpde_observables_noalloc(const dpde_params* params, const dpde_replica* replica, const double* q,
                             const double* p, const double* eps, void* stream, dpde_obs* out) {
    g_na_error.clear();
    if (!params || !replica || !out) return na_fail(DPDE_ERR_ARG, "params, replica and out are required");
    const dpde_params& P = *params;
    const dpde_replica& Rp = *replica;
    if (!(P.mass > 0) || !(P.r_cut > 0) || !(P.a >= 0) || !(Rp.cv > 0) || Rp.n < 0 ||
        (Rp.walls != 0 && Rp.walls != 1) ||
        (P.potential != DPDE_POT_SOFT && P.potential != DPDE_POT_LJ) ||
        (P.potential == DPDE_POT_LJ && (!(P.lj_eps >= 0) || !(P.lj_r > 0))))
        return na_fail(DPDE_ERR_ARG, "invalid parameters");
    if (Rp.n > NA_MAX_N)
        return na_fail(DPDE_ERR_ARG, "dpde_observables_noalloc: n = " + std::to_string(Rp.n) +
                                         " exceeds the fixed scratch limit of " + std::to_string(NA_MAX_N) +
                                         " particles");
    if (Rp.n > 0 && (!q || !p || !eps)) return na_fail(DPDE_ERR_ARG, "q, p and eps are required");
    NaGeom G{};
    long long ncells = 1;
    for (int d = 0; d < 3; ++d) {
        if (!(Rp.box[d] > 0)) return na_fail(DPDE_ERR_ARG, "invalid box");
        G.L[d] = Rp.box[d];
        G.nc[d] = (int)std::floor(Rp.box[d] / P.r_cut);
        if (G.nc[d] < 3) return na_fail(DPDE_ERR_ARG, "box shorter than 3 r_cut along an axis");
        G.s[d] = (double)G.nc[d] / Rp.box[d];
        ncells *= G.nc[d];
    }
    if (ncells > NA_MAX_CELLS)
        return na_fail(DPDE_ERR_ARG, "dpde_observables_noalloc: " + std::to_string(ncells) +
                                         " cells exceed the fixed scratch limit of " +
                                         std::to_string(NA_MAX_CELLS));
    G.rc = P.r_cut;
    G.rc2 = P.r_cut * P.r_cut;
    G.a = P.a;
    G.pot = dpde::make_pot(P.potential, P.a, P.r_cut, P.lj_eps, P.lj_r);
    G.mass = P.mass;
    G.cv = Rp.cv;
    G.n = (int)Rp.n;
    G.walls = Rp.walls;
    // device address of the scratch array, looked up once per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(DPDE_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(DPDE_ERR_ARG, "device index out of range");
    if (G.n > 0) {
        const void* ptrs[3] = {q, p, eps};
        const char* names[3] = {"q", "p", "eps"};
        for (int k = 0; k < 3; ++k) {
            const int rc = na_check_device_ptr(ptrs[k], dev, names[k]);
            if (rc != DPDE_OK) return rc;
        }
    }
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess)
                return na_fail(DPDE_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_na_ptr[dev] = (unsigned char*)ptr;
        }
        base = g_na_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    int* count = (int*)(base + OFF_COUNT);
    int* start = (int*)(base + OFF_START);
    int* fill = (int*)(base + OFF_FILL);
    int* perm = (int*)(base + OFF_PERM);
    double* partial = (double*)(base + OFF_PART);
    double* res = (double*)(base + OFF_OUT);
    // the array keeps the previous call's contents: clear what must start at zero
    e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)ncells, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(fill, 0, sizeof(int) * (size_t)ncells, st);
    if (e != cudaSuccess) return na_fail(DPDE_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int nb = (G.n + NA_THREADS - 1) / NA_THREADS;
    if (G.n > 0) {
        k_na_count<<<nb, NA_THREADS, 0, st>>>(G, q, count);
        k_na_scan<<<1, NA_THREADS, 0, st>>>(count, start, (int)ncells);
        k_na_scatter<<<nb, NA_THREADS, 0, st>>>(G, q, start, fill, perm);
    }
    k_na_terms<<<NA_BLOCKS, NA_THREADS, 0, st>>>(G, q, p, eps, start, perm, partial);
    k_na_final<<<1, 32, 0, st>>>(partial, res);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(DPDE_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    double t[NA_TERMS];
    e = cudaMemcpyAsync(t, res, sizeof(t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return na_fail(DPDE_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(e));
    const long long n = G.n;
    std::memset(out, 0, sizeof(*out));
    out->K = t[0]; out->U = t[1]; out->Eint = t[2];
    out->E = out->U + out->K + out->Eint;
    out->P[0] = t[3]; out->P[1] = t[4]; out->P[2] = t[5];
    out->Tkin = n > 1 ? 2.0 * out->K / (3.0 * (double)(n - 1)) : 0.0;
    out->Tint = n > 0 ? (double)n / t[6] : 0.0;
    out->Tpot_num = t[7];
    out->Tpot_den = t[8];
    out->n = n;
    out->neg_eps = (int64_t)t[9];
    out->nonfinite = (int64_t)t[10];
    if (out->nonfinite > 0) return na_fail(DPDE_ERR_NONFINITE, "non-finite value in the state");
    if (out->neg_eps > 0) return na_fail(DPDE_ERR_NEG_EPS, "internal energy eps_i <= 0");
    return DPDE_OK;
}

const char* dpde_noalloc_last_error(void) { return g_na_error.c_str(); }

}  // extern "C"
