// dpde_api.cu -- the C ABI of include/dpde.h: handle, buffers, launch
// sequence of one timestep, CUDA-graph replay, observables, diagnostics.
#include "dpde.h"
#include "dpde_ssa_levels.cuh"
#include "dpde_ssa_persistent.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

using namespace dpde;

namespace {

// A named NVTX range over the body of a C-ABI call (header-only NVTX v3: no
// cost and no dependency unless a profiler is attached), so that profilers
// can attribute work to the entry point that issued it.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

thread_local std::string g_create_error;

int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

struct GraphKey {
    int scheme;
    unsigned long long dt_bits;
    bool operator<(const GraphKey& o) const {
        return scheme != o.scheme ? scheme < o.scheme : dt_bits < o.dt_bits;
    }
};

}  // namespace

constexpr int STATE_CHUNKS = 4;   // chunks of a host <-> device state transfer

struct dpde_handle {
    dpde_params prm{};
    int R = 0;
    std::vector<dpde_replica> reps;
    std::vector<RepInfo> info;
    int N = 0;
    int ncells = 0;
    int nbricks = 0;
    int nchunks = 0;
    int nbr_cap = 0;
    bool mixed = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;
    // host <-> device state transfers: copies on their own stream, in chunks,
    // overlapping the conversion kernels of the neighbouring chunks
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t xfer_ev[STATE_CHUNKS + 1] = {};
    cudaStream_t ssa_stream = nullptr;       // the SSA schedule's deferred launches
    cudaEvent_t ssa_ev[2] = {};
    // device buffers
    void *qA = nullptr, *pA = nullptr, *qB = nullptr, *pB = nullptr, *F = nullptr, *dp = nullptr;
    void* upot = nullptr;            // per-particle potential energy share (T)
    // projection on the internal energies (Sec. IV.C)
    bool project = false;
    double *proj_e0 = nullptr, *proj_shift = nullptr, *proj_partial = nullptr;
    void *eA = nullptr, *eB = nullptr, *nbr_w = nullptr, *fwd_w = nullptr, *fwd_g = nullptr;
    int *cA = nullptr, *cB = nullptr, *nbr_j = nullptr, *nbr_n = nullptr, *fwd_j = nullptr, *fwd_n = nullptr;
    int4 *tile_org = nullptr, *tile_dim = nullptr;
    int ntiles = 0;
    // SSA colour classes: cells grouped by colour index (col_z * 5 + col_y) * 5
    // + col_x, for the brick domains (Hybrid) and the whole replica (SSA)
    int* col_cells[2] = {nullptr, nullptr};
    std::vector<int> col_off[2];   // NCOLOURS + 1 offsets into col_cells
    // SSA domain by domain (ssa_mode 1, Hybrid): the cells of each brick
    // sorted by colour class, and per brick the NCOLOURS + 1 class starts
    int* dom_cells = nullptr;
    int* dom_off = nullptr;
    int* dom_cell0 = nullptr;    // first cell of each brick, then ncells
    double dom_mean = 0.0;       // most particles per brick of a replica, on average
    int ssa_mode = 2;
    bool any_walls = false;       // some replica has walls along z
    WallPos* wallpos = nullptr;   // upper wall of each replica for the step's drift
    // SSA by dependency levels (ssa_mode 2): domain tables of whole replicas
    // (DPDE_SSA; the bricks' are dom_*), per-domain level offsets and counts,
    // the deferred-domain lists ([0] schedule count, [1] execution count,
    // then the two lists), and the shared-memory capacities per table
    int *rdom_cells = nullptr, *rdom_off = nullptr, *rdom_cell0 = nullptr;
    int *lv_off = nullptr, *lv_n = nullptr, *ssa_defer = nullptr;
    int ndom_max = 1;
    struct SsaCaps {
        // three tiers each: regular (one block per domain), deferred (a few
        // blocks per SM), large (one block per SM)
        int scap_s[3] = {0, 0, 0}, ecap_s[3] = {0, 0, 0}, ccap_s[3] = {0, 0, 0}, scap_x[3] = {0, 0, 0};
        int grid_s[3] = {0, 0, 0}, grid_x[3] = {0, 0, 0};
        bool ok = false;   // domains small enough for the level form
    } ssa_caps[2];
    int nsm = 152;
    // the persistent per-class SSA launch (ssa_mode 3): class offsets on the
    // device, its grid barrier and the barrier's wait budget (clock cycles)
    int* d_col_off[2] = {nullptr, nullptr};
    GridBarrier* d_bar = nullptr;
    long long wait_budget = 2000000000ll;
    int ssa_group = 0;        // bricks per warp; 0 = dom_group_auto
    int dom_group_auto = 1;   // 32 / the largest class of a brick, in 1..SSA_GROUP_MAX
    int hcap = 0;             // halo particles staged per force tile
    int hcap_dense = 0;       // ... per deferred (dense) tile
    size_t tile_smem_dense = 0;
    int* defer = nullptr;     // deferred tiles of the force pass: list, then count
    int ndense_blocks = 0;
    int hcc = 0;              // halo cells per force tile, (tile_edge + 2)^3
    size_t tile_smem = 0;
    double per_cell_max = 0;  // mean particles per cell of the densest replica
    // tuning (dpde_set_tuning / dpde_autotune)
    int tile_edge = TILE_EDGE;
    int ssa_block = SSA_THREADS;
    uint32_t* idB = nullptr;
    int *key = nullptr, *tmp = nullptr, *cnt = nullptr, *start = nullptr, *bsum = nullptr;
    int *rep_of_slot = nullptr, *rep_of_cell = nullptr, *brick_rep = nullptr, *tab = nullptr;
    int *chunk_rep = nullptr, *chunk_begin = nullptr, *chunk_end = nullptr, *rep_chunk_begin = nullptr;
    double *partial = nullptr, *obs_out = nullptr;
    RepInfo* d_reps = nullptr;
    long long* d_step = nullptr;
    unsigned int* d_status = nullptr;
    double* staging = nullptr;       // 7N doubles: q (3N), p (3N), eps (N)
    int* cells_out = nullptr;        // 3N ints (diagnostic)
    long long step = 0;              // host mirror of the device counter
    int block = 256;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    cudaEvent_t prof_ev[DPDE_NUM_PHASES][2] = {};
    bool profiling = false;
    bool prof_used[DPDE_NUM_PHASES] = {};
    std::string err;
};

namespace {

int fail(dpde_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(dpde_handle* h, cudaError_t e, const char* what) {
    return fail(h, e == cudaErrorMemoryAllocation ? DPDE_ERR_OOM : DPDE_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                                  \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);     \
    } while (0)

template <class T>
Ctx<T> make_ctx(dpde_handle* h) {
    Ctx<T> C;
    using vec = vec_t<T>;
    using E = eps_t<T>;
    C.qA = (vec*)h->qA; C.pA = (vec*)h->pA; C.eA = (E*)h->eA; C.cA = h->cA;
    C.qB = (vec*)h->qB; C.pB = (vec*)h->pB; C.eB = (E*)h->eB; C.cB = h->cB;
    C.idB = h->idB;
    C.F = (vec*)h->F; C.dp = (vec*)h->dp;
    C.upot = (T*)h->upot;
    C.key = h->key; C.tmp = h->tmp;
    C.count = h->cnt; C.fill = h->cnt + h->ncells; C.start = h->start;
    C.nbr_j = h->nbr_j; C.nbr_w = (T*)h->nbr_w; C.nbr_n = h->nbr_n; C.nbr_cap = h->nbr_cap;
    C.fwd_j = h->fwd_j; C.fwd_w = (T*)h->fwd_w; C.fwd_g = (vec_t<T>*)h->fwd_g; C.fwd_n = h->fwd_n;
    C.rep_of_slot = h->rep_of_slot; C.rep_of_cell = h->rep_of_cell;
    C.brick_rep = h->brick_rep; C.tab = h->tab;
    C.reps = h->d_reps; C.step = h->d_step; C.status = h->d_status; C.wall = h->wallpos;
    C.N = h->N; C.ncells = h->ncells;
    C.m = (T)h->prm.mass; C.inv_m = (T)(1.0 / h->prm.mass);
    C.rc = (T)h->prm.r_cut; C.rc2 = (T)(h->prm.r_cut * h->prm.r_cut);
    C.inv_rc = (T)(1.0 / h->prm.r_cut);
    C.a = (T)h->prm.a; C.sigma = (T)h->prm.sigma;
    C.pot = cast_pot<T>(make_pot(h->prm.potential, h->prm.a, h->prm.r_cut, h->prm.lj_eps, h->prm.lj_r));
    C.sig2_4 = (T)(h->prm.sigma * h->prm.sigma / 4.0);
    C.seed = make_uint2((uint32_t)(h->prm.seed & 0xffffffffu), (uint32_t)(h->prm.seed >> 32));
    return C;
}

// The level form's records live in the buffer of the forward entries'
// Gaussians (unused by that form): N * cap 32-bit (s, t) words, then, from a
// 256-byte boundary, N * cap weights.
size_t ssa_rec_w_offset(const dpde_handle* h) {
    return ((size_t)std::max(1, h->N) * (size_t)h->nbr_cap * sizeof(uint32_t) + 255) & ~(size_t)255;
}

// phase markers (only when dpde_step_profiled is running)
void phase(dpde_handle* h, cudaStream_t st, int ph, int end) {
    if (!h->profiling) return;
    cudaEventRecord(h->prof_ev[ph][end], st);
    h->prof_used[ph] = true;
}

// cell sort of set A into set B (kick = 1: Verlet first half before it)
template <class T>
void enqueue_sort(dpde_handle* h, const Ctx<T>& C, cudaStream_t st, T half_dt, T dt, int kick) {
    const int nb = ceil_div(h->N, h->block);
    phase(h, st, DPDE_PHASE_KICK_DRIFT, 0);
    cudaMemsetAsync(h->cnt, 0, sizeof(int) * 2 * (size_t)h->ncells, st);
    k_kick_drift_key<T><<<nb, h->block, 0, st>>>(C, half_dt, dt, kick);
    phase(h, st, DPDE_PHASE_KICK_DRIFT, 1);
    phase(h, st, DPDE_PHASE_SCAN, 0);
    const int ntile = ceil_div(h->ncells, SCAN_TILE);
    k_scan_local<<<ntile, SCAN_THREADS, 0, st>>>(h->cnt, h->start, h->bsum, h->ncells);
    k_scan_bsums<<<1, 1024, 0, st>>>(h->bsum, ntile);
    k_scan_add<<<ceil_div(h->ncells, 256), 256, 0, st>>>(h->start, h->bsum, h->ncells, h->N);
    phase(h, st, DPDE_PHASE_SCAN, 1);
    phase(h, st, DPDE_PHASE_GATHER, 0);
    k_scatter<T><<<nb, h->block, 0, st>>>(C);
    k_rank_gather<T><<<nb, h->block, 0, st>>>(C);
    phase(h, st, DPDE_PHASE_GATHER, 1);
}

template <class T>
void enqueue_force(dpde_handle* h, const Ctx<T>& C, cudaStream_t st, T half_dt, int kick, int list) {
    const dim3 g(h->ntiles), blk(TILE_THREADS), gd(h->ndense_blocks);
    int* cnt = h->defer + h->ntiles;
    cudaMemsetAsync(cnt, 0, sizeof(int), st);
#define DPDE_FORCE(LMV)                                                                                          \
    k_force_tile<T, LMV><<<g, blk, h->tile_smem, st>>>(C, h->tile_org, h->tile_dim, half_dt, kick, h->hcap,      \
                                                       h->hcc, h->defer, cnt);                                   \
    k_force_tile_dense<T, LMV><<<gd, blk, h->tile_smem_dense, st>>>(C, h->tile_org, h->tile_dim, half_dt, kick, \
                                                                    h->hcap_dense, h->hcc, h->defer, cnt)
    switch (list) {
    case LIST_ALL: DPDE_FORCE(LIST_ALL); break;
    case LIST_CROSS: DPDE_FORCE(LIST_CROSS); break;
    case LIST_FWD: DPDE_FORCE(LIST_FWD); break;
    default: DPDE_FORCE(LIST_NONE); break;
    }
#undef DPDE_FORCE
}

// The SSA sequence: the Gaussians of every forward entry, then either, for
// brick domains (Hybrid, ssa_mode 1), one launch in which each warp walks the
// colour classes of whole bricks, or one launch per non-empty colour class,
// in colour order; both apply the same sequence.
// The SSA sequence by dependency levels (ssa_mode 2): the schedule of every
// domain, then its execution; each kernel's regular launch (one block per
// domain) defers domains beyond its shared-memory capacities to a second,
// persistent launch with larger ones. The domains the schedule's regular
// launch defers (the large ones of an uneven batch or a shock front) are
// scheduled and then executed on a second stream, beside the execution's
// regular launch, which leaves them alone: the two streams touch disjoint
// domains, and the long chains of the large ones start before the many small
// ones are done.
template <class T>
void enqueue_ssa_levels(dpde_handle* h, const Ctx<T>& C, cudaStream_t st, T dt, T sqrt_dt, int whole) {
    const dpde_handle::SsaCaps& K = h->ssa_caps[whole];
    const SsaDomains D = whole ? SsaDomains{h->rdom_cells, h->rdom_off, h->rdom_cell0, h->R}
                               : SsaDomains{h->dom_cells, h->dom_off, h->dom_cell0, h->nbricks};
    SsaLevels<T> V;
    V.lv_off = h->lv_off;
    V.lv_n = h->lv_n;
    V.rec_st = reinterpret_cast<uint32_t*>(h->fwd_g);
    V.rec_w = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(h->fwd_g) + ssa_rec_w_offset(h));
    // counts: [0, 1] schedule tiers 1, 2; [2, 3] execution tiers 1, 2 of the
    // domains the regular schedule kept; [4, 5] execution tiers 1, 2 of those
    // it deferred; then the lists
    int* cnt = h->ssa_defer;
    int* lst[SSA_NLISTS];
    for (int k = 0; k < SSA_NLISTS; ++k) lst[k] = cnt + SSA_NLISTS + (size_t)k * h->ndom_max;
    cudaMemsetAsync(cnt, 0, SSA_NLISTS * sizeof(int), st);
    auto sched_tiers = [&](cudaStream_t s) {
        for (int t = 1; t < 3; ++t)
            k_ssa_sched<T><<<K.grid_s[t], SCHED_THREADS, ssa_sched_smem(K.scap_s[t], K.ecap_s[t], K.ccap_s[t]),
                             s>>>(C, D, V, K.scap_s[t], K.ecap_s[t], K.ccap_s[t], 0, lst[t - 1], cnt + t - 1,
                                  t < 2 ? lst[t] : nullptr, t < 2 ? cnt + t : nullptr);
    };
    // execution tiers 1, 2 over the list at index l0 (tier 1) and l0 + 1 (tier 2)
    auto exec_tiers = [&](cudaStream_t s, int* first, int* nfirst, int l1) {
        k_ssa_exec<T><<<K.grid_x[1], h->ssa_block, ssa_exec_smem<T>(K.scap_x[1]), s>>>(
            C, D, V, K.scap_x[1], 0, first, nfirst, lst[l1], cnt + l1, dt, sqrt_dt);
        k_ssa_exec<T><<<K.grid_x[2], h->ssa_block, ssa_exec_smem<T>(K.scap_x[2]), s>>>(
            C, D, V, K.scap_x[2], 0, lst[l1], cnt + l1, nullptr, nullptr, dt, sqrt_dt);
    };
    auto sched_regular = [&](cudaStream_t s, int d0, int n) {
        k_ssa_sched<T><<<n, SCHED_THREADS, ssa_sched_smem(K.scap_s[0], K.ecap_s[0], K.ccap_s[0]), s>>>(
            C, D, V, K.scap_s[0], K.ecap_s[0], K.ccap_s[0], d0, nullptr, nullptr, lst[0], cnt);
    };
    auto exec_regular = [&](cudaStream_t s, int d0, int n) {
        k_ssa_exec<T><<<n, h->ssa_block, ssa_exec_smem<T>(K.scap_x[0]), s>>>(C, D, V, K.scap_x[0], d0, nullptr,
                                                                             nullptr, lst[2], cnt + 2, dt, sqrt_dt);
    };
    if (h->profiling) {   // phase by phase, one stream
        phase(h, st, DPDE_PHASE_SSA_GAUSS, 0);
        sched_regular(st, 0, D.n);
        sched_tiers(st);
        phase(h, st, DPDE_PHASE_SSA_GAUSS, 1);
        phase(h, st, DPDE_PHASE_SSA, 0);
        exec_regular(st, 0, D.n);
        exec_tiers(st, lst[2], cnt + 2, 3);
        exec_tiers(st, lst[0], cnt, 4);
        phase(h, st, DPDE_PHASE_SSA, 1);
        return;
    }
    sched_regular(st, 0, D.n);
    cudaEventRecord(h->ssa_ev[0], st);
    cudaStreamWaitEvent(h->ssa_stream, h->ssa_ev[0], 0);
    sched_tiers(h->ssa_stream);                       // the deferred domains: scheduled,
    exec_tiers(h->ssa_stream, lst[0], cnt, 4);        // then executed
    exec_regular(st, 0, D.n);                         // the others, beside them
    exec_tiers(st, lst[2], cnt + 2, 3);
    cudaEventRecord(h->ssa_ev[1], h->ssa_stream);
    cudaStreamWaitEvent(st, h->ssa_ev[1], 0);
}

template <class T>
void enqueue_ssa(dpde_handle* h, const Ctx<T>& C, cudaStream_t st, T dt, T sqrt_dt, int whole) {
    if (h->ssa_mode == 2 && h->ssa_caps[whole].ok) {
        enqueue_ssa_levels<T>(h, C, st, dt, sqrt_dt, whole);
        return;
    }
    const std::vector<int>& off = h->col_off[whole];
    phase(h, st, DPDE_PHASE_SSA_GAUSS, 0);
    k_ssa_gauss<T><<<ceil_div(h->N, 256), 256, 0, st>>>(C);
    phase(h, st, DPDE_PHASE_SSA_GAUSS, 1);
    phase(h, st, DPDE_PHASE_SSA, 0);
    if (!whole && h->ssa_mode == 1 && h->nbricks > 0) {
        const int group = h->ssa_group > 0 ? h->ssa_group : h->dom_group_auto;
        const int warps = ceil_div(h->nbricks, group);
        // one warp per block: the warps share nothing, and single-warp blocks
        // pack the staged shared memory without splitting a wave
        const int wpb = 1;
        // staged slots per warp: the group's mean particle count + 25 % + 64,
        // as far as the shared memory of a block allows
        const size_t per_slot = sizeof(vec_t<T>) + sizeof(eps_t<T>);
        const size_t fixed = ssa_domain_warp_bytes<T>(group, 0);
        long long scap = ((long long)std::ceil(1.25 * group * h->dom_mean) + 64 + 31) / 32 * 32;
        const long long fit = ((long long)(SSA_DOMAIN_SMEM / wpb) - (long long)fixed) / (long long)per_slot;
        scap = std::max(0ll, std::min(scap, fit / 32 * 32));
        k_ssa_domains<T><<<ceil_div(warps, wpb), 32 * wpb, wpb * ssa_domain_warp_bytes<T>(group, (int)scap), st>>>(
            C, h->dom_cells, h->dom_off, h->dom_cell0, h->nbricks, group, (int)scap, dt, sqrt_dt);
        phase(h, st, DPDE_PHASE_SSA, 1);
        return;
    }
    if (h->ssa_mode == 3) {
        // one cooperative launch over all classes, a grid barrier between them
        const size_t smem = ssa_smem_bytes(h->ssa_block);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ssa_persistent<T>, h->ssa_block, smem);
        cudaMemsetAsync(h->d_bar, 0, sizeof(GridBarrier), st);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)std::max(1, per_sm * h->nsm));
        cfg.blockDim = dim3((unsigned)h->ssa_block);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, k_ssa_persistent<T>, C, (const int*)h->col_cells[whole],
                           (const int*)h->d_col_off[whole], dt, sqrt_dt, h->d_bar, h->wait_budget);
        phase(h, st, DPDE_PHASE_SSA, 1);
        return;
    }
    for (int k = 0; k < NCOLOURS; ++k) {
        const int n = off[k + 1] - off[k];
        if (n > 0)
            k_ssa_colour<T><<<ceil_div(n, h->ssa_block), h->ssa_block, ssa_smem_bytes(h->ssa_block), st>>>(
                C, h->col_cells[whole] + off[k], n, dt, sqrt_dt);
    }
    phase(h, st, DPDE_PHASE_SSA, 1);
}

template <class T>
void enqueue_step(dpde_handle* h, cudaStream_t st, double dt_d, int scheme) {
    const Ctx<T> C = make_ctx<T>(h);
    const T dt = (T)dt_d, half_dt = (T)(0.5 * dt_d), sqrt_dt = (T)std::sqrt(dt_d);
    if (h->any_walls) k_wall_pos<T><<<ceil_div(h->R, 64), 64, 0, st>>>(C, h->R, dt_d);
    const int nb = ceil_div(h->N, h->block);
    enqueue_sort<T>(h, C, st, half_dt, dt, 1);
    const int list = scheme == DPDE_SSA ? LIST_FWD : (scheme == DPDE_HYBRID ? LIST_CROSS : LIST_ALL);
    phase(h, st, DPDE_PHASE_FORCE, 0);
    enqueue_force<T>(h, C, st, half_dt, 1, list);
    phase(h, st, DPDE_PHASE_FORCE, 1);
    if (scheme == DPDE_HYBRID || scheme == DPDE_SSA) {
        enqueue_ssa<T>(h, C, st, dt, sqrt_dt, scheme == DPDE_SSA ? 1 : 0);
    }
    if (scheme == DPDE_SER || scheme == DPDE_HYBRID) {
        phase(h, st, DPDE_PHASE_SWEEP1, 0);
        k_ser_sweep1<T><<<nb, h->block, 0, st>>>(C, dt, sqrt_dt);
        phase(h, st, DPDE_PHASE_SWEEP1, 1);
    }
    phase(h, st, DPDE_PHASE_SWEEP2, 0);
    if (scheme == DPDE_SER || scheme == DPDE_HYBRID) k_ser_sweep2<T><<<nb, h->block, 0, st>>>(C, dt, sqrt_dt);
    else if (scheme == DPDE_SEM) k_sem<T><<<nb, h->block, 0, st>>>(C, dt, sqrt_dt);
    else k_copy_back<T><<<nb, h->block, 0, st>>>(C);
    phase(h, st, DPDE_PHASE_SWEEP2, 1);
    if (h->project) {
        phase(h, st, DPDE_PHASE_OTHER, 0);
        if (h->nchunks > 0)
            k_proj_chunks<T><<<h->nchunks, OBS_THREADS, 0, st>>>(C, h->chunk_begin, h->chunk_end, h->proj_partial);
        k_proj_reps<T><<<ceil_div(h->R, 128), 128, 0, st>>>(C, h->proj_partial, h->rep_chunk_begin, h->R,
                                                             h->proj_e0, h->proj_shift);
        k_proj_apply<T><<<nb, h->block, 0, st>>>(C, h->proj_shift);
        phase(h, st, DPDE_PHASE_OTHER, 1);
    }
    k_step_inc<<<1, 1, 0, st>>>(h->d_step);
}

// Rebuilds the cell starts of the current A set (already in (cell, id) order)
// without moving anything: the keys come from the stored cells and the
// gather into B is the identity. Needed after the A set is written directly.
void enqueue_rebin(dpde_handle* h, cudaStream_t st) {
    if (h->mixed) enqueue_sort<float>(h, make_ctx<float>(h), st, 0.f, 0.f, 0);
    else enqueue_sort<double>(h, make_ctx<double>(h), st, 0.0, 0.0, 0);
}

void enqueue_step_any(dpde_handle* h, cudaStream_t st, double dt, int scheme) {
    if (h->mixed) enqueue_step<float>(h, st, dt, scheme);
    else enqueue_step<double>(h, st, dt, scheme);
}

// The state in: from device arrays, or from host arrays copied into the
// staging buffer chunk by chunk on the copy stream, each chunk converted as
// soon as it has arrived.
template <class T>
void enqueue_set_state(dpde_handle* h, cudaStream_t st, const double* q, const double* p, const double* e,
                       bool host) {
    const Ctx<T> C = make_ctx<T>(h);
    const long long N = h->N;
    const int nb = ceil_div(h->N, h->block);
    const int K = host && N >= (1 << 16) ? STATE_CHUNKS : 1;
    const double *dq = q, *dp = p, *de = e;
    if (host) {
        dq = h->staging; dp = h->staging + 3 * N; de = h->staging + 6 * N;
        cudaEventRecord(h->xfer_ev[STATE_CHUNKS], st);   // the staging buffer is free
        cudaStreamWaitEvent(h->copy_stream, h->xfer_ev[STATE_CHUNKS], 0);
    }
    for (int c = 0; c < K; ++c) {
        const long long s0 = N * c / K, s1 = N * (c + 1) / K;
        if (s1 == s0) continue;
        if (host) {
            const size_t n = (size_t)(s1 - s0);
            cudaMemcpyAsync(h->staging + 3 * s0, q + 3 * s0, sizeof(double) * 3 * n, cudaMemcpyHostToDevice,
                            h->copy_stream);
            cudaMemcpyAsync(h->staging + 3 * N + 3 * s0, p + 3 * s0, sizeof(double) * 3 * n,
                            cudaMemcpyHostToDevice, h->copy_stream);
            cudaMemcpyAsync(h->staging + 6 * N + s0, e + s0, sizeof(double) * n, cudaMemcpyHostToDevice,
                            h->copy_stream);
            cudaEventRecord(h->xfer_ev[c], h->copy_stream);
            cudaStreamWaitEvent(st, h->xfer_ev[c], 0);
        }
        k_load_state<T><<<ceil_div((int)(s1 - s0), h->block), h->block, 0, st>>>(C, dq, dp, de, (int)s0, (int)s1);
    }
    enqueue_sort<T>(h, C, st, T(0), T(0), 0);
    enqueue_force<T>(h, C, st, T(0), 0, LIST_NONE);
    k_copy_back<T><<<nb, h->block, 0, st>>>(C);
}

// The state out: into device arrays, or into host arrays through the
// staging buffer, each chunk of ids copied while the next is gathered; st
// waits for the copies at the end.
template <class T>
void enqueue_get_state(dpde_handle* h, cudaStream_t st, double* q, double* p, double* e, bool host) {
    const Ctx<T> C = make_ctx<T>(h);
    const long long N = h->N;
    // the sort's scratch (tmp, N ints) holds the id -> slot map between steps
    k_slot_of_id<T><<<ceil_div(h->N, h->block), h->block, 0, st>>>(C, h->tmp);
    const int K = host && N >= (1 << 16) ? STATE_CHUNKS : 1;
    double* dq = host ? (q ? h->staging : nullptr) : q;
    double* dp = host ? (p ? h->staging + 3 * N : nullptr) : p;
    double* de = host ? (e ? h->staging + 6 * N : nullptr) : e;
    for (int c = 0; c < K; ++c) {
        const long long g0 = N * c / K, g1 = N * (c + 1) / K;
        if (g1 == g0) continue;
        k_get_state<T><<<ceil_div((int)(g1 - g0), h->block), h->block, 0, st>>>(C, h->tmp, dq, dp, de, (int)g0,
                                                                              (int)g1);
        if (host) {
            const size_t n = (size_t)(g1 - g0);
            cudaEventRecord(h->xfer_ev[c], st);
            cudaStreamWaitEvent(h->copy_stream, h->xfer_ev[c], 0);
            if (q) cudaMemcpyAsync(q + 3 * g0, dq + 3 * g0, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost,
                                   h->copy_stream);
            if (p) cudaMemcpyAsync(p + 3 * g0, dp + 3 * g0, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost,
                                   h->copy_stream);
            if (e) cudaMemcpyAsync(e + g0, de + g0, sizeof(double) * n, cudaMemcpyDeviceToHost, h->copy_stream);
        }
    }
    if (host) {
        cudaEventRecord(h->xfer_ev[STATE_CHUNKS], h->copy_stream);
        cudaStreamWaitEvent(st, h->xfer_ev[STATE_CHUNKS], 0);
    }
}

template <class T>
void enqueue_obs(dpde_handle* h, cudaStream_t st) {
    const Ctx<T> C = make_ctx<T>(h);
    if (h->nchunks > 0)
        k_obs_chunks<T><<<h->nchunks, OBS_THREADS, 0, st>>>(C, h->chunk_rep, h->chunk_begin, h->chunk_end,
                                                             h->partial);
    k_obs_reps<<<h->R, 32, 0, st>>>(h->partial, h->rep_chunk_begin, h->R, h->obs_out);
}

int read_status(dpde_handle* h) {
    unsigned int st = 0;
    CK(h, cudaMemcpyAsync(&st, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (st & ST_TIMEOUT)
        return fail(h, DPDE_ERR_TIMEOUT, "a grid barrier of the persistent SSA launch waited past its budget; "
                                         "the step's state is incomplete");
    if (st & ST_CAPACITY) return fail(h, DPDE_ERR_CAPACITY, "neighbour list capacity exceeded");
    if (st & ST_WALL) return fail(h, DPDE_ERR_ARG, "the moving wall reached the lowest cell layer");
    if (st & ST_DOMAIN) return fail(h, DPDE_ERR_CUDA, "internal error: an SSA chain left its domain");
    if (st & ST_NONFINITE) return fail(h, DPDE_ERR_NONFINITE, "non-finite value in the state");
    if (st & ST_NEG_EPS) return fail(h, DPDE_ERR_NEG_EPS, "internal energy eps_i <= 0");
    return DPDE_OK;
}

void free_all(dpde_handle* h) {
    for (auto& row : h->prof_ev)
        for (auto& ev : row)
            if (ev) cudaEventDestroy(ev);
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    void* bufs[] = {h->qA, h->pA, h->qB, h->pB, h->F, h->dp, h->upot, h->proj_e0, h->proj_shift, h->proj_partial, h->eA, h->eB, h->nbr_w, h->cA, h->cB, h->nbr_j,
                    h->nbr_n, h->fwd_j, h->fwd_w, h->fwd_g, h->fwd_n, h->tile_org, h->tile_dim, h->defer, h->col_cells[0], h->col_cells[1], h->dom_cells, h->dom_off, h->dom_cell0, h->rdom_cells, h->rdom_off, h->rdom_cell0, h->lv_off, h->lv_n, h->ssa_defer, h->d_col_off[0], h->d_col_off[1], h->d_bar, h->wallpos, h->idB, h->key, h->tmp, h->cnt, h->start, h->bsum, h->rep_of_slot,
                    h->rep_of_cell, h->brick_rep, h->tab, h->chunk_rep, h->chunk_begin, h->chunk_end,
                    h->rep_chunk_begin, h->partial, h->obs_out, h->d_reps, h->d_step, h->d_status,
                    h->staging, h->cells_out};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->ssa_stream) cudaStreamDestroy(h->ssa_stream);
    for (auto& ev : h->ssa_ev)
        if (ev) cudaEventDestroy(ev);
    for (auto& ev : h->xfer_ev)
        if (ev) cudaEventDestroy(ev);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

// Force tiles of edge `edge` cells over every replica, their halo staging
// capacity (1.08x the mean halo count of the densest replica + 64, over 3
// standard deviations of a uniform fluid's count) and shared memory size.
int set_tiles(dpde_handle* h, int edge) {
    std::vector<int4> torg, tdim;
    for (int r = 0; r < h->R; ++r) {
        const RepInfo& I = h->info[r];
        for (int z0 = 0; z0 < I.nc[2]; z0 += edge)
            for (int y0 = 0; y0 < I.nc[1]; y0 += edge)
                for (int x0 = 0; x0 < I.nc[0]; x0 += edge) {
                    torg.push_back(make_int4(r, x0, y0, z0));
                    tdim.push_back(make_int4(std::min(edge, I.nc[0] - x0), std::min(edge, I.nc[1] - y0),
                                             std::min(edge, I.nc[2] - z0), 0));
                }
    }
    const int hcc = (edge + 2) * (edge + 2) * (edge + 2);
    const size_t thead = tile_head_bytes(hcc);
    const size_t tper = h->mixed ? tile_per_particle<float>() : tile_per_particle<double>();
    const double mean_halo = h->per_cell_max * hcc;
    const size_t smem_limit = 200 * 1024;
    int hcap = (int)std::min<double>(std::min<double>(1.08 * mean_halo + 64.0, 65535.0),
                                     (double)((smem_limit - thead) / tper));
    hcap &= ~3;   // keeps the arrays after the positions 16-byte aligned
    const size_t smem = 32 + thead + (size_t)hcap * tper;
    // deferred tiles: 2.5x the mean halo (dense regions such as a shock front)
    int hcap_dense = (int)std::min<double>(std::min<double>(2.5 * mean_halo + 64.0, 65535.0),
                                           (double)((smem_limit + 24 * 1024 - thead) / tper));
    hcap_dense = std::max(hcap_dense, hcap) & ~3;
    const size_t smem_dense = 32 + thead + (size_t)hcap_dense * tper;
    if (h->tile_org) cudaFree(h->tile_org);
    if (h->tile_dim) cudaFree(h->tile_dim);
    if (h->defer) cudaFree(h->defer);
    h->tile_org = h->tile_dim = nullptr;
    h->defer = nullptr;
    CK(h, cudaMalloc(&h->defer, sizeof(int) * (torg.size() + 1)));
    CK(h, cudaMalloc(&h->tile_org, sizeof(int4) * std::max<size_t>(1, torg.size())));
    CK(h, cudaMalloc(&h->tile_dim, sizeof(int4) * std::max<size_t>(1, tdim.size())));
    CK(h, cudaMemcpy(h->tile_org, torg.data(), sizeof(int4) * torg.size(), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->tile_dim, tdim.data(), sizeof(int4) * tdim.size(), cudaMemcpyHostToDevice));
    const int sm = (int)smem, smd = (int)smem_dense;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (h->mixed) {
        CK(h, cudaFuncSetAttribute(k_force_tile<float, LIST_NONE>, A, sm));
        CK(h, cudaFuncSetAttribute(k_force_tile<float, LIST_ALL>, A, sm));
        CK(h, cudaFuncSetAttribute(k_force_tile<float, LIST_CROSS>, A, sm));
        CK(h, cudaFuncSetAttribute(k_force_tile<float, LIST_FWD>, A, sm));
        CK(h, cudaFuncSetAttribute(k_force_tile_dense<float, LIST_NONE>, A, smd));
        CK(h, cudaFuncSetAttribute(k_force_tile_dense<float, LIST_ALL>, A, smd));
        CK(h, cudaFuncSetAttribute(k_force_tile_dense<float, LIST_CROSS>, A, smd));
        CK(h, cudaFuncSetAttribute(k_force_tile_dense<float, LIST_FWD>, A, smd));
    } else {
        CK(h, cudaFuncSetAttribute(k_force_tile<double, LIST_NONE>, A, sm));
        CK(h, cudaFuncSetAttribute(k_force_tile<double, LIST_ALL>, A, sm));
        CK(h, cudaFuncSetAttribute(k_force_tile<double, LIST_CROSS>, A, sm));
        CK(h, cudaFuncSetAttribute(k_force_tile<double, LIST_FWD>, A, sm));
        CK(h, cudaFuncSetAttribute(k_force_tile_dense<double, LIST_NONE>, A, smd));
        CK(h, cudaFuncSetAttribute(k_force_tile_dense<double, LIST_ALL>, A, smd));
        CK(h, cudaFuncSetAttribute(k_force_tile_dense<double, LIST_CROSS>, A, smd));
        CK(h, cudaFuncSetAttribute(k_force_tile_dense<double, LIST_FWD>, A, smd));
    }
    h->ntiles = (int)torg.size();
    h->hcc = hcc;
    h->hcap = hcap;
    h->tile_smem = smem;
    h->hcap_dense = hcap_dense;
    h->tile_smem_dense = smem_dense;
    int nsm = 152;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    h->ndense_blocks = std::max(1, std::min((int)torg.size(), nsm));
    h->tile_edge = edge;
    return DPDE_OK;
}

}  // namespace

extern "C" {

int dpde_create(const dpde_params* params, int32_t n_replicas, const dpde_replica* replicas,
                void* stream, dpde_handle** out) {
    NvtxRange nvtx_range_("dpde_create");
    g_create_error.clear();
    if (!out) return fail(nullptr, DPDE_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!params || !replicas || n_replicas < 1) return fail(nullptr, DPDE_ERR_ARG, "bad params/replicas");
    const dpde_params& P = *params;
    if (!(P.mass > 0) || !(P.r_cut > 0) || !(P.a >= 0) || !(P.sigma >= 0) ||
        (P.potential != DPDE_POT_SOFT && P.potential != DPDE_POT_LJ) ||
        (P.potential == DPDE_POT_LJ && (!(P.lj_eps >= 0) || !(P.lj_r > 0) || !std::isfinite(P.lj_eps) ||
                                        !std::isfinite(P.lj_r))) ||
        (P.precision != DPDE_FP64 && P.precision != DPDE_MIXED))
        return fail(nullptr, DPDE_ERR_ARG, "invalid dpde_params");
    dpde_handle* h = new dpde_handle();
    h->prm = P;
    h->R = n_replicas;
    h->mixed = P.precision == DPDE_MIXED;
    h->reps.assign(replicas, replicas + n_replicas);
    long long N = 0, ncells = 0, nbricks = 0;
    const int CHUNK = 4096;
    std::vector<int> chunk_rep, chunk_begin, chunk_end, rep_chunk_begin(1, 0), tabs, brick_rep;
    double rho_max = 0.0, per_cell_max = 0.0;
    for (int r = 0; r < n_replicas; ++r) {
        const dpde_replica& d = replicas[r];
        RepInfo I{};
        if (d.n < 0 || !(d.cv > 0)) {
            delete h;
            return fail(nullptr, DPDE_ERR_ARG, "replica " + std::to_string(r) + ": bad n/cv");
        }
        if ((d.walls != 0 && d.walls != 1) || (d.walls == 1 && !(d.wall_u <= 0.0))) {
            delete h;
            return fail(nullptr, DPDE_ERR_ARG, "replica " + std::to_string(r) + ": walls must be 0 or 1, wall_u <= 0");
        }
        for (int a = 0; a < 3; ++a) {
            if (!(d.box[a] > 0) || d.bricks[a] < 1) {
                delete h;
                return fail(nullptr, DPDE_ERR_ARG, "replica " + std::to_string(r) + ": bad box/bricks");
            }
            I.k[a] = (int)std::floor(d.box[a] / ((double)d.bricks[a] * P.r_cut));
            I.B[a] = d.bricks[a];
            I.nc[a] = I.B[a] * I.k[a];
            if (I.k[a] < 1 || I.nc[a] < 3 || I.nc[a] > 1024) {
                delete h;
                return fail(nullptr, DPDE_ERR_ARG,
                            "replica " + std::to_string(r) + ": box does not fit the brick grid (need "
                            "floor(L/(B r_cut)) >= 1 and 3 <= B*that <= 1024 cells per axis)");
            }
            I.L[a] = d.box[a];
            I.ell[a] = d.box[a] / (double)I.nc[a];
            I.s[a] = (double)I.nc[a] / d.box[a];
            I.ellf[a] = (float)I.ell[a];
        }
        const int kc = I.k[0] * I.k[1] * I.k[2];
        const int nbr = I.B[0] * I.B[1] * I.B[2];
        I.cell_off = (int)ncells;
        I.ncells = I.nc[0] * I.nc[1] * I.nc[2];
        I.part_off = (int)N;
        I.n = (int)d.n;
        I.brick_off = (int)nbricks;
        I.tab_off = (int)tabs.size();
        I.cv = d.cv;
        I.cvf = (float)d.cv;
        I.walls = d.walls;
        I.wall_u = d.walls ? d.wall_u : 0.0;
        h->any_walls = h->any_walls || d.walls;
        // brick-major cell tables
        for (int c = 0; c < I.nc[0]; ++c) tabs.push_back((c / I.k[0]) * kc + c % I.k[0]);
        for (int c = 0; c < I.nc[1]; ++c) tabs.push_back((c / I.k[1]) * I.B[0] * kc + (c % I.k[1]) * I.k[0]);
        for (int c = 0; c < I.nc[2]; ++c)
            tabs.push_back((c / I.k[2]) * I.B[0] * I.B[1] * kc + (c % I.k[2]) * I.k[0] * I.k[1]);
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < I.nc[a]; ++c) tabs.push_back(c / I.k[a]);
        for (int b = 0; b < nbr; ++b) brick_rep.push_back(r);
        per_cell_max = std::max(per_cell_max, (double)d.n / (double)(I.nc[0] * I.nc[1] * I.nc[2]));
        rho_max = std::max(rho_max, (double)d.n / (d.box[0] * d.box[1] * d.box[2]));
        h->info.push_back(I);
        N += d.n;
        ncells += I.ncells;
        nbricks += nbr;
        for (long long b = 0; b < d.n; b += CHUNK) {
            chunk_rep.push_back(r);
            chunk_begin.push_back((int)(I.part_off + b));
            chunk_end.push_back((int)(I.part_off + std::min<long long>(b + CHUNK, d.n)));
        }
        rep_chunk_begin.push_back((int)chunk_rep.size());
        if (N > (1ll << NBR_J_BITS) || ncells > (1ll << 30)) {
            delete h;
            return fail(nullptr, DPDE_ERR_ARG, "too many particles (limit 2^27) or cells (2^30)");
        }
    }
    h->N = (int)N;
    h->ncells = (int)ncells;
    h->nbricks = (int)nbricks;
    h->nchunks = (int)chunk_rep.size();
    h->per_cell_max = per_cell_max;
    // neighbour-list capacity: 3x the mean neighbour count of the densest replica, + 32
    const double mean_nbr = 4.0 / 3.0 * M_PI * rho_max * P.r_cut * P.r_cut * P.r_cut;
    h->nbr_cap = (int)std::ceil(3.0 * mean_nbr) + 32;
    const size_t vsz = h->mixed ? sizeof(float4) : sizeof(d4);
    const size_t esz = h->mixed ? sizeof(ff) : sizeof(double);
    // SSA colour classes (cell colours of the SSA order, per axis l mod P
    // with P = 3, 3, 2 along x, y, z, and colours P, P + 1 for the last
    // k mod P cells of a periodic domain axis), for brick domains (m = 0)
    // and whole replicas (m = 1)
    std::vector<int> col_cells[2];
    std::vector<unsigned char> dom_col((size_t)std::max<long long>(1, ncells), 0);
    std::vector<unsigned char> rep_col((size_t)std::max<long long>(1, ncells), 0);
    for (int m = 0; m < 2; ++m) {
        std::vector<std::vector<int>> cls(NCOLOURS);
        for (const RepInfo& I : h->info) {
            const int* tx = tabs.data() + I.tab_off;
            const int* ty = tx + I.nc[0];
            const int* tz = ty + I.nc[1];
            int col[3][1024];
            for (int a = 0; a < 3; ++a) {
                const bool periodic = (m == 1 || I.B[a] == 1) && !(a == 2 && I.walls);
                const int k = m == 1 ? I.nc[a] : I.k[a];
                const int P = a == 2 ? 2 : 3;
                const int full = P * (k / P);
                for (int c = 0; c < I.nc[a]; ++c) {
                    const int l = m == 1 ? c : c % I.k[a];
                    col[a][c] = (periodic && l >= full) ? P + (l - full) : l % P;
                }
            }
            for (int z = 0; z < I.nc[2]; ++z)
                for (int y = 0; y < I.nc[1]; ++y)
                    for (int x = 0; x < I.nc[0]; ++x) {
                        const int k = (col[2][z] * 5 + col[1][y]) * 5 + col[0][x];
                        const int c = I.cell_off + tx[x] + ty[y] + tz[z];
                        cls[k].push_back(c);
                        (m == 0 ? dom_col : rep_col)[c] = (unsigned char)k;
                    }
        }
        h->col_off[m].assign(1, 0);
        for (auto& v : cls) {
            std::sort(v.begin(), v.end());
            col_cells[m].insert(col_cells[m].end(), v.begin(), v.end());
            h->col_off[m].push_back((int)col_cells[m].size());
        }
    }
    // per brick (brick-major cell order: brick b of replica I holds cells
    // cell_off + b k_x k_y k_z onwards) its cells sorted by colour class
    std::vector<int> dom_cells, dom_off, dom_cell0;
    dom_cells.reserve((size_t)ncells);
    dom_off.reserve((size_t)nbricks * (NCOLOURS + 1));
    int class_max = 1;
    for (const RepInfo& I : h->info) {
        const int kc = I.k[0] * I.k[1] * I.k[2];
        const int nbr = I.B[0] * I.B[1] * I.B[2];
        h->dom_mean = std::max(h->dom_mean, (double)I.n / nbr);
        for (int b = 0; b < nbr; ++b) {
            int cnt[NCOLOURS + 1] = {0};
            const int c0 = I.cell_off + b * kc;
            dom_cell0.push_back(c0);
            for (int c = c0; c < c0 + kc; ++c) ++cnt[dom_col[c] + 1];
            const int base = (int)dom_cells.size();
            dom_off.push_back(base);
            for (int k = 0; k < NCOLOURS; ++k) {
                class_max = std::max(class_max, cnt[k + 1]);
                cnt[k + 1] += cnt[k];
                dom_off.push_back(base + cnt[k + 1]);
            }
            dom_cells.resize(dom_cells.size() + kc);
            for (int c = c0; c < c0 + kc; ++c) dom_cells[base + cnt[dom_col[c]]++] = c;
        }
    }
    dom_cell0.push_back((int)ncells);
    h->dom_group_auto = std::max(1, std::min(SSA_GROUP_MAX, 32 / class_max));
    // the same per whole replica (the domain of DPDE_SSA)
    std::vector<int> rdom_cells, rdom_off, rdom_cell0;
    rdom_cells.reserve((size_t)ncells);
    for (const RepInfo& I : h->info) {
        int cnt[NCOLOURS + 1] = {0};
        const int c0 = I.cell_off;
        rdom_cell0.push_back(c0);
        for (int c = c0; c < c0 + I.ncells; ++c) ++cnt[rep_col[c] + 1];
        const int base = (int)rdom_cells.size();
        rdom_off.push_back(base);
        for (int k = 0; k < NCOLOURS; ++k) {
            cnt[k + 1] += cnt[k];
            rdom_off.push_back(base + cnt[k + 1]);
        }
        rdom_cells.resize(rdom_cells.size() + I.ncells);
        for (int c = c0; c < c0 + I.ncells; ++c) rdom_cells[base + cnt[rep_col[c]]++] = c;
    }
    rdom_cell0.push_back((int)ncells);
    // shared-memory capacities of the level form, per domain table (0 bricks,
    // 1 whole replicas), from the mean domain size M, in three tiers: the
    // regular launches (a block per domain) hold M + 5 sqrt(M) + 32
    // particles (a uniform fluid's domains stay below) for the execution,
    // 1.3 M + 64 particles and 1.2 M e + 256 entries (e forward entries per
    // particle at the densest replica's density) for the schedule; the
    // deferred launches (several blocks per SM) ~2.5x that; the last ones
    // what ~200 KB hold. The form is used where no domain is expected above
    // 16,384 particles.
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
        const double e_pp = 2.0 / 3.0 * M_PI * rho_max * P.r_cut * P.r_cut * P.r_cut * 1.15;
        const size_t smem_big = 200 * 1024;
        const size_t per = h->mixed ? (sizeof(float4) + sizeof(ff) + 4) : (sizeof(d4) + sizeof(double) + 4);
        for (int t = 0; t < 2; ++t) {
            dpde_handle::SsaCaps& K = h->ssa_caps[t];
            const int ndom = t == 0 ? (int)nbricks : n_replicas;
            double biggest = 0.0;
            for (const RepInfo& I : h->info)
                biggest = std::max(biggest, t == 0 ? (double)I.n / (I.B[0] * I.B[1] * I.B[2]) : (double)I.n);
            const double M = ndom > 0 ? (double)N / ndom : 0.0;
            auto up16 = [](double x) { return ((int)std::ceil(x) + 15) / 16 * 16; };
            // entries that fit beside sc particles in ~200 KB of schedule
            auto ecap_fit = [&](int sc, int cc) {
                return std::min(SSA_LOCAL_MAX,
                                (int)((smem_big - (SSA_LV_STRIDE + cc) * sizeof(int)) / 2 - (2 * sc + 1)) / 16 * 16);
            };
            // schedule: 1.3 M particles / 1.2 M e entries; 2.5 M / 6.25 M e (a
            // brick compressed 2.5-fold holds ~6x the entries) in ~96 KB; the
            // largest that ~200 KB hold. Cell ranges staged for up to half as
            // many cells as particles (density 3 has a third) in the first two.
            K.scap_s[0] = std::min(16384, up16(1.3 * M + 64));
            K.ccap_s[0] = K.scap_s[0] / 2;
            K.ecap_s[0] = std::min(ecap_fit(K.scap_s[0], K.ccap_s[0]), up16(1.2 * M * e_pp + 256));
            K.scap_s[1] = std::min(16384, up16(2.5 * M + 64));
            K.ccap_s[1] = K.scap_s[1] / 2;
            K.ecap_s[1] = std::min(ecap_fit(K.scap_s[1], K.ccap_s[1]), up16(6.25 * M * e_pp + 256));
            while (K.ecap_s[1] > K.ecap_s[0] &&
                   ssa_sched_smem(K.scap_s[1], K.ecap_s[1], K.ccap_s[1]) > smem_big / 2)
                K.ecap_s[1] = std::max(K.ecap_s[0], K.ecap_s[1] * 7 / 8 / 16 * 16);
            K.scap_s[2] = 16384;
            K.ccap_s[2] = 0;
            K.ecap_s[2] = ecap_fit(K.scap_s[2], 0);
            // execution: M + 5 sqrt(M) + 32 particles; 2.5 M in <= 96 KB; ~200 KB
            const int xfit = (int)((smem_big - 32) / per);
            K.scap_x[0] = std::min(xfit, ((int)std::ceil(M + 5.0 * std::sqrt(M) + 32) + 31) / 32 * 32);
            K.scap_x[1] = std::max(K.scap_x[0], std::min(xfit / 2, ((int)std::ceil(2.5 * M + 64) + 31) / 32 * 32));
            K.scap_x[2] = xfit;
            const size_t smem_sm = 227 * 1024;
            K.grid_s[0] = ndom;
            K.grid_s[1] = h->nsm * std::max<int>(1, (int)(smem_sm / (ssa_sched_smem(K.scap_s[1], K.ecap_s[1],
                                                                                      K.ccap_s[1]) + 1024)));
            K.grid_s[2] = h->nsm;
            K.grid_x[0] = ndom;
            const size_t xs1 = h->mixed ? ssa_exec_smem<float>(K.scap_x[1]) : ssa_exec_smem<double>(K.scap_x[1]);
            K.grid_x[1] = h->nsm * std::max<int>(1, std::min<int>(8, (int)(smem_sm / (xs1 + 1024))));
            K.grid_x[2] = h->nsm;
            K.ok = biggest <= 16384.0;
        }
    }
    auto bail = [&](cudaError_t e, const char* what) {
        std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
        int code = e == cudaErrorMemoryAllocation ? DPDE_ERR_OOM : DPDE_ERR_CUDA;
        free_all(h);
        delete h;
        return fail(nullptr, code, msg);
    };
#define CKC(call)                                      \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return bail(e_, #call); \
    } while (0)
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        CKC(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    CKC(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CKC(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    for (auto& ev : h->xfer_ev) CKC(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CKC(cudaStreamCreateWithFlags(&h->ssa_stream, cudaStreamNonBlocking));
    for (auto& ev : h->ssa_ev) CKC(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    const size_t n1 = (size_t)std::max(1, h->N), c1 = (size_t)std::max(1, h->ncells);
    const size_t tsz = h->mixed ? sizeof(float) : sizeof(double);
    CKC(cudaMalloc(&h->qA, vsz * n1));
    CKC(cudaMalloc(&h->pA, vsz * n1));
    CKC(cudaMalloc(&h->qB, vsz * n1));
    CKC(cudaMalloc(&h->pB, vsz * n1));
    CKC(cudaMalloc(&h->F, vsz * n1));
    CKC(cudaMalloc(&h->dp, vsz * n1));
    CKC(cudaMalloc(&h->upot, tsz * n1));
    CKC(cudaMalloc(&h->proj_e0, sizeof(double) * (size_t)h->R));
    CKC(cudaMalloc(&h->proj_shift, sizeof(double) * (size_t)h->R));
    CKC(cudaMalloc(&h->proj_partial, sizeof(double) * std::max<size_t>(1, chunk_rep.size())));
    CKC(cudaMalloc(&h->eA, esz * n1));
    CKC(cudaMalloc(&h->eB, esz * n1));
    CKC(cudaMalloc(&h->cA, sizeof(int) * n1));
    CKC(cudaMalloc(&h->cB, sizeof(int) * n1));
    CKC(cudaMalloc(&h->idB, sizeof(uint32_t) * n1));
    CKC(cudaMalloc(&h->nbr_j, sizeof(int) * n1 * (size_t)h->nbr_cap));
    CKC(cudaMalloc(&h->nbr_w, tsz * n1 * (size_t)h->nbr_cap));
    CKC(cudaMalloc(&h->nbr_n, sizeof(int) * n1));
    CKC(cudaMalloc(&h->fwd_j, sizeof(int) * n1 * (size_t)h->nbr_cap));
    CKC(cudaMalloc(&h->fwd_w, tsz * n1 * (size_t)h->nbr_cap));
    CKC(cudaMalloc(&h->fwd_g, vsz * n1 * (size_t)h->nbr_cap));
    CKC(cudaMalloc(&h->fwd_n, sizeof(int) * n1));
    CKC(cudaMalloc(&h->key, sizeof(int) * n1));
    CKC(cudaMalloc(&h->tmp, sizeof(int) * n1));
    CKC(cudaMalloc(&h->cnt, sizeof(int) * 2 * c1));
    CKC(cudaMalloc(&h->start, sizeof(int) * (c1 + 1)));
    CKC(cudaMalloc(&h->bsum, sizeof(int) * (size_t)std::max(1, ceil_div(h->ncells, SCAN_TILE))));
    CKC(cudaMalloc(&h->rep_of_slot, sizeof(int) * n1));
    CKC(cudaMalloc(&h->rep_of_cell, sizeof(int) * c1));
    CKC(cudaMalloc(&h->brick_rep, sizeof(int) * (size_t)std::max(1, h->nbricks)));
    CKC(cudaMalloc(&h->tab, sizeof(int) * tabs.size()));
    CKC(cudaMalloc(&h->chunk_rep, sizeof(int) * std::max<size_t>(1, chunk_rep.size())));
    CKC(cudaMalloc(&h->chunk_begin, sizeof(int) * std::max<size_t>(1, chunk_rep.size())));
    CKC(cudaMalloc(&h->chunk_end, sizeof(int) * std::max<size_t>(1, chunk_rep.size())));
    CKC(cudaMalloc(&h->rep_chunk_begin, sizeof(int) * rep_chunk_begin.size()));
    CKC(cudaMalloc(&h->partial, sizeof(double) * NTERMS * std::max<size_t>(1, chunk_rep.size())));
    CKC(cudaMalloc(&h->obs_out, sizeof(double) * NTERMS * (size_t)h->R));
    CKC(cudaMalloc(&h->d_reps, sizeof(RepInfo) * (size_t)h->R));
    CKC(cudaMalloc(&h->wallpos, sizeof(WallPos) * (size_t)std::max(1, h->R)));
    CKC(cudaMalloc(&h->d_step, sizeof(long long)));
    CKC(cudaMalloc(&h->d_status, sizeof(unsigned int)));
    CKC(cudaMalloc(&h->staging, sizeof(double) * 7 * n1));
    CKC(cudaMalloc(&h->cells_out, sizeof(int) * 3 * n1));
    {
        std::vector<int> ros(n1, 0), roc(c1, 0);
        for (int r = 0; r < h->R; ++r) {
            const RepInfo& I = h->info[r];
            for (int s = 0; s < I.n; ++s) ros[I.part_off + s] = r;
            for (int c = 0; c < I.ncells; ++c) roc[I.cell_off + c] = r;
        }
        CKC(cudaMemcpy(h->rep_of_slot, ros.data(), sizeof(int) * n1, cudaMemcpyHostToDevice));
        CKC(cudaMemcpy(h->rep_of_cell, roc.data(), sizeof(int) * c1, cudaMemcpyHostToDevice));
        CKC(cudaMemcpy(h->brick_rep, brick_rep.data(), sizeof(int) * brick_rep.size(), cudaMemcpyHostToDevice));
        CKC(cudaMemcpy(h->tab, tabs.data(), sizeof(int) * tabs.size(), cudaMemcpyHostToDevice));
        if (!chunk_rep.empty()) {
            CKC(cudaMemcpy(h->chunk_rep, chunk_rep.data(), sizeof(int) * chunk_rep.size(), cudaMemcpyHostToDevice));
            CKC(cudaMemcpy(h->chunk_begin, chunk_begin.data(), sizeof(int) * chunk_rep.size(), cudaMemcpyHostToDevice));
            CKC(cudaMemcpy(h->chunk_end, chunk_end.data(), sizeof(int) * chunk_rep.size(), cudaMemcpyHostToDevice));
        }
        CKC(cudaMemcpy(h->rep_chunk_begin, rep_chunk_begin.data(), sizeof(int) * rep_chunk_begin.size(),
                       cudaMemcpyHostToDevice));
        CKC(cudaMemcpy(h->d_reps, h->info.data(), sizeof(RepInfo) * (size_t)h->R, cudaMemcpyHostToDevice));
        CKC(cudaMemset(h->d_step, 0, sizeof(long long)));
        CKC(cudaMemset(h->d_status, 0, sizeof(unsigned int)));
        CKC(cudaMemset(h->eA, 0, esz * n1));
        CKC(cudaMemset(h->qA, 0, vsz * n1));
        CKC(cudaMemset(h->pA, 0, vsz * n1));
        CKC(cudaMemset(h->cA, 0, sizeof(int) * n1));
        CKC(cudaMemset(h->F, 0, vsz * n1));
        CKC(cudaMemset(h->nbr_n, 0, sizeof(int) * n1));
        CKC(cudaMemset(h->fwd_n, 0, sizeof(int) * n1));
    }
    CKC(cudaMalloc(&h->dom_cells, sizeof(int) * std::max<size_t>(1, dom_cells.size())));
    CKC(cudaMalloc(&h->dom_off, sizeof(int) * std::max<size_t>(1, dom_off.size())));
    if (!dom_cells.empty())
        CKC(cudaMemcpy(h->dom_cells, dom_cells.data(), sizeof(int) * dom_cells.size(), cudaMemcpyHostToDevice));
    if (!dom_off.empty())
        CKC(cudaMemcpy(h->dom_off, dom_off.data(), sizeof(int) * dom_off.size(), cudaMemcpyHostToDevice));
    CKC(cudaMalloc(&h->dom_cell0, sizeof(int) * dom_cell0.size()));
    CKC(cudaMemcpy(h->dom_cell0, dom_cell0.data(), sizeof(int) * dom_cell0.size(), cudaMemcpyHostToDevice));
    CKC(cudaMalloc(&h->rdom_cells, sizeof(int) * std::max<size_t>(1, rdom_cells.size())));
    CKC(cudaMalloc(&h->rdom_off, sizeof(int) * rdom_off.size()));
    CKC(cudaMalloc(&h->rdom_cell0, sizeof(int) * rdom_cell0.size()));
    if (!rdom_cells.empty())
        CKC(cudaMemcpy(h->rdom_cells, rdom_cells.data(), sizeof(int) * rdom_cells.size(), cudaMemcpyHostToDevice));
    CKC(cudaMemcpy(h->rdom_off, rdom_off.data(), sizeof(int) * rdom_off.size(), cudaMemcpyHostToDevice));
    CKC(cudaMemcpy(h->rdom_cell0, rdom_cell0.data(), sizeof(int) * rdom_cell0.size(), cudaMemcpyHostToDevice));
    h->ndom_max = std::max(1, std::max(h->nbricks, h->R));
    CKC(cudaMalloc(&h->lv_off, sizeof(int) * (size_t)h->ndom_max * SSA_LV_STRIDE));
    CKC(cudaMalloc(&h->lv_n, sizeof(int) * (size_t)h->ndom_max));
    CKC(cudaMalloc(&h->ssa_defer, sizeof(int) * (SSA_NLISTS + SSA_NLISTS * (size_t)h->ndom_max)));
    {
        size_t ms = 0, mx = 0;
        for (const auto& K : h->ssa_caps)
            for (int t = 0; t < 3; ++t) {
                ms = std::max(ms, ssa_sched_smem(K.scap_s[t], K.ecap_s[t], K.ccap_s[t]));
                mx = std::max(mx, h->mixed ? ssa_exec_smem<float>(K.scap_x[t]) : ssa_exec_smem<double>(K.scap_x[t]));
            }
        const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if (h->mixed) {
            CKC(cudaFuncSetAttribute(k_ssa_sched<float>, A, (int)ms));
            CKC(cudaFuncSetAttribute(k_ssa_exec<float>, A, (int)mx));
        } else {
            CKC(cudaFuncSetAttribute(k_ssa_sched<double>, A, (int)ms));
            CKC(cudaFuncSetAttribute(k_ssa_exec<double>, A, (int)mx));
        }
    }
    if (h->mixed)
        CKC(cudaFuncSetAttribute(k_ssa_domains<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, SSA_DOMAIN_SMEM));
    else
        CKC(cudaFuncSetAttribute(k_ssa_domains<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, SSA_DOMAIN_SMEM));
    CKC(cudaMalloc(&h->d_bar, sizeof(GridBarrier)));
    CKC(cudaMemset(h->d_bar, 0, sizeof(GridBarrier)));
    for (int m = 0; m < 2; ++m) {
        CKC(cudaMalloc(&h->d_col_off[m], sizeof(int) * (NCOLOURS + 1)));
        CKC(cudaMemcpy(h->d_col_off[m], h->col_off[m].data(), sizeof(int) * (NCOLOURS + 1), cudaMemcpyHostToDevice));
        CKC(cudaMalloc(&h->col_cells[m], sizeof(int) * c1));
        if (!col_cells[m].empty())
            CKC(cudaMemcpy(h->col_cells[m], col_cells[m].data(), sizeof(int) * col_cells[m].size(),
                           cudaMemcpyHostToDevice));
    }
    {
        const int rc = set_tiles(h, TILE_EDGE);
        if (rc != DPDE_OK) {
            const std::string msg = h->err;
            free_all(h);
            delete h;
            return fail(nullptr, rc, msg);
        }
    }
#undef CKC
    *out = h;
    return DPDE_OK;
}

int dpde_set_state(dpde_handle* h, const double* q, const double* p, const double* eps, int64_t step,
                   int32_t on_device) {
    NvtxRange nvtx_range_("dpde_set_state");
    if (!h) return DPDE_ERR_ARG;
    if (h->N > 0 && (!q || !p || !eps)) return fail(h, DPDE_ERR_ARG, "q, p and eps are required");
    const size_t N = (size_t)h->N;
    CK(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), h->stream));
    if (N > 0) {
        if (h->mixed) enqueue_set_state<float>(h, h->stream, q, p, eps, !on_device);
        else enqueue_set_state<double>(h, h->stream, q, p, eps, !on_device);
    }
    long long s = step;
    CK(h, cudaMemcpyAsync(h->d_step, &s, sizeof(long long), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaGetLastError());
    h->step = step;
    return read_status(h);
}

int dpde_get_state(dpde_handle* h, double* q, double* p, double* eps, int32_t on_device) {
    NvtxRange nvtx_range_("dpde_get_state");
    if (!h) return DPDE_ERR_ARG;
    const size_t N = (size_t)h->N;
    if (N > 0) {
        if (h->mixed) enqueue_get_state<float>(h, h->stream, q, p, eps, !on_device);
        else enqueue_get_state<double>(h, h->stream, q, p, eps, !on_device);
        CK(h, cudaGetLastError());
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return read_status(h);
}

int dpde_get_cells(dpde_handle* h, int32_t* cells) {
    if (!h || (h->N > 0 && !cells)) return DPDE_ERR_ARG;
    if (h->N > 0) {
        if (h->mixed) k_get_cells<float><<<ceil_div(h->N, h->block), h->block, 0, h->stream>>>(make_ctx<float>(h), h->cells_out);
        else k_get_cells<double><<<ceil_div(h->N, h->block), h->block, 0, h->stream>>>(make_ctx<double>(h), h->cells_out);
        CK(h, cudaGetLastError());
        CK(h, cudaMemcpyAsync(cells, h->cells_out, sizeof(int) * 3 * (size_t)h->N, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return DPDE_OK;
}

int dpde_step(dpde_handle* h, int64_t n, double dt, int32_t scheme, int32_t use_graph) {
    NvtxRange nvtx_range_("dpde_step");
    if (!h) return DPDE_ERR_ARG;
    if (n < 0 || !(dt > 0) || !std::isfinite(dt) || scheme < DPDE_SER || scheme > DPDE_SSA)
        return fail(h, DPDE_ERR_ARG, "bad n, dt or scheme");
    if (n == 0 || h->N == 0) {
        h->step += n;
        if (n > 0) {
            long long s = h->step;
            CK(h, cudaMemcpyAsync(h->d_step, &s, sizeof(long long), cudaMemcpyHostToDevice, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
        }
        return DPDE_OK;
    }
    if (use_graph) {
        GraphKey gk{scheme, 0};
        std::memcpy(&gk.dt_bits, &dt, sizeof(double));
        auto it = h->graphs.find(gk);
        if (it == h->graphs.end()) {
            cudaGraph_t g = nullptr;
            CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
            enqueue_step_any(h, h->cap_stream, dt, scheme);
            CK(h, cudaStreamEndCapture(h->cap_stream, &g));
            cudaGraphExec_t ex = nullptr;
            cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
            it = h->graphs.emplace(gk, ex).first;
        }
        for (int64_t k = 0; k < n; ++k) CK(h, cudaGraphLaunch(it->second, h->stream));
    } else {
        for (int64_t k = 0; k < n; ++k) enqueue_step_any(h, h->stream, dt, scheme);
        CK(h, cudaGetLastError());
    }
    h->step += n;
    return DPDE_OK;
}

int dpde_set_projection(dpde_handle* h, int32_t enable, const double* E0) {
    if (!h || (enable != 0 && enable != 1)) return DPDE_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    if (!enable) {
        h->project = false;
        return DPDE_OK;
    }
    std::vector<double> e0((size_t)h->R);
    if (E0) {
        for (int r = 0; r < h->R; ++r) {
            if (!std::isfinite(E0[r])) return fail(h, DPDE_ERR_ARG, "E0 must be finite");
            e0[r] = E0[r];
        }
    } else {
        std::vector<dpde_obs> obs((size_t)h->R);
        const int rc = dpde_observables(h, obs.data());
        if (rc != DPDE_OK && rc != DPDE_ERR_NEG_EPS) return rc;
        for (int r = 0; r < h->R; ++r) e0[r] = obs[r].E;
    }
    CK(h, cudaMemcpy(h->proj_e0, e0.data(), sizeof(double) * (size_t)h->R, cudaMemcpyHostToDevice));
    h->project = true;
    return DPDE_OK;
}

int dpde_set_wait_budget(dpde_handle* h, int64_t cycles) {
    if (!h) return DPDE_ERR_ARG;
    if (cycles < 0) return fail(h, DPDE_ERR_ARG, "the wait budget must be >= 0 clock cycles");
    CK(h, cudaStreamSynchronize(h->stream));
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    h->wait_budget = cycles;
    return DPDE_OK;
}

int dpde_get_tuning(dpde_handle* h, dpde_tuning* out) {
    if (!h || !out) return DPDE_ERR_ARG;
    out->tile_edge = h->tile_edge;
    out->block = h->block;
    out->ssa_block = h->ssa_block;
    out->ssa_mode = h->ssa_mode;
    out->ssa_group = h->ssa_group > 0 ? h->ssa_group : h->dom_group_auto;
    out->reserved = 0;
    out->ms_per_step = 0.0;
    return DPDE_OK;
}

int dpde_set_tuning(dpde_handle* h, const dpde_tuning* t) {
    if (!h || !t) return DPDE_ERR_ARG;
    if (t->tile_edge < 2 || t->tile_edge > TILE_EDGE_MAX || t->block < 64 || t->block > 1024 ||
        t->block % 32 != 0 || t->ssa_block < 32 || t->ssa_block > SSA_THREADS_MAX || t->ssa_block % 32 != 0 ||
        (t->ssa_mode < 0 || t->ssa_mode > 3) || t->ssa_group < 0 || t->ssa_group > SSA_GROUP_MAX ||
        t->reserved != 0)
        return fail(h, DPDE_ERR_ARG, "tuning out of range");
    CK(h, cudaStreamSynchronize(h->stream));
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    if (t->tile_edge != h->tile_edge) {
        const int rc = set_tiles(h, t->tile_edge);
        if (rc != DPDE_OK) return rc;
    }
    h->block = t->block;
    h->ssa_block = t->ssa_block;
    h->ssa_mode = t->ssa_mode;
    h->ssa_group = t->ssa_group;
    return DPDE_OK;
}

int dpde_autotune(dpde_handle* h, int32_t scheme, double dt, int32_t steps, dpde_tuning* out) {
    NvtxRange nvtx_range_("dpde_autotune");
    if (!h) return DPDE_ERR_ARG;
    if (scheme < DPDE_SER || scheme > DPDE_SSA || !(dt > 0) || !std::isfinite(dt) || steps < 1 || steps > 1000)
        return fail(h, DPDE_ERR_ARG, "bad scheme, dt or steps");
    dpde_tuning best{};
    dpde_get_tuning(h, &best);
    if (h->N == 0) {
        if (out) *out = best;
        return DPDE_OK;
    }
    // saved state: A set, forces, step counter
    const size_t n = (size_t)h->N;
    const size_t vsz = h->mixed ? sizeof(float4) : sizeof(d4);
    const size_t esz = h->mixed ? sizeof(ff) : sizeof(double);
    const size_t bytes = 3 * vsz * n + esz * n + sizeof(int) * n + sizeof(long long);
    unsigned char* save = nullptr;
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMalloc(&save, bytes));
    struct Piece { void* dev; size_t size; };
    const Piece pieces[] = {{h->qA, vsz * n}, {h->pA, vsz * n}, {h->F, vsz * n}, {h->eA, esz * n},
                            {h->cA, sizeof(int) * n}, {h->d_step, sizeof(long long)}};
    auto copy_all = [&](bool to_save) -> cudaError_t {
        size_t off = 0;
        for (const Piece& pc : pieces) {
            cudaError_t e = to_save ? cudaMemcpyAsync(save + off, pc.dev, pc.size, cudaMemcpyDeviceToDevice, h->stream)
                                    : cudaMemcpyAsync(pc.dev, save + off, pc.size, cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) return e;
            off += pc.size;
        }
        return cudaSuccess;
    };
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int rc = DPDE_OK;
    // one trial: the step captured as a graph (as dpde_step runs it), one
    // untimed replay, then `steps` timed replays
    auto trial = [&](const dpde_tuning& t, double& ms) -> int {
        int r = dpde_set_tuning(h, &t);
        if (r != DPDE_OK) return r;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ex = nullptr;
        CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        enqueue_step_any(h, h->cap_stream, dt, scheme);
        CK(h, cudaStreamEndCapture(h->cap_stream, &g));
        const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return cuda_fail(h, ie, "cudaGraphInstantiate");
        cudaError_t e = cudaGraphLaunch(ex, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], h->stream);
        for (int k = 0; k < steps && e == cudaSuccess; ++k) e = cudaGraphLaunch(ex, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        cudaGraphExecDestroy(ex);
        if (e != cudaSuccess) return cuda_fail(h, e, "autotune trial");
        float f = 0.f;
        CK(h, cudaEventElapsedTime(&f, ev[0], ev[1]));
        ms = (double)f / steps;
        CK(h, copy_all(false));
        CK(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        return DPDE_OK;
    };
    do {
        if ((rc = (cudaEventCreate(&ev[0]) == cudaSuccess && cudaEventCreate(&ev[1]) == cudaSuccess)
                      ? DPDE_OK : fail(h, DPDE_ERR_CUDA, "cudaEventCreate")) != DPDE_OK)
            break;
        if (copy_all(true) != cudaSuccess) { rc = fail(h, DPDE_ERR_CUDA, "saving the state"); break; }
        double best_ms = 0.0;
        if ((rc = trial(best, best_ms)) != DPDE_OK) break;
        const int edges[] = {4, 5, 6, 7, 8}, blocks[] = {128, 256, 512}, ssa_blocks[] = {32, 64, 128},
                  modes[] = {2, 1, 0, 3}, groups[] = {1, 2, 3, 4};
        const int* cands[] = {edges, blocks, ssa_blocks, modes, groups};
        const int ncands[] = {5, 3, 3, 4, 4};
        for (int stage = 0; stage < 5 && rc == DPDE_OK; ++stage) {
            // bricks per warp matter only to the per-brick SSA launch
            if (stage == 4 && (best.ssa_mode != 1 || scheme != DPDE_HYBRID)) break;
            const int* cand = cands[stage];
            const int nc = ncands[stage];
            dpde_tuning base = best;
            for (int c = 0; c < nc && rc == DPDE_OK; ++c) {
                dpde_tuning t = base;
                int* field[] = {&t.tile_edge, &t.block, &t.ssa_block, &t.ssa_mode, &t.ssa_group};
                *field[stage] = cand[c];
                double ms = 0.0;
                rc = trial(t, ms);
                // a candidate must beat the incumbent by more than the trial noise
                if (rc == DPDE_OK && ms < 0.99 * best_ms) {
                    best_ms = ms;
                    best = t;
                }
            }
        }
        if (rc != DPDE_OK) break;
        best.ms_per_step = 0.0;
        if ((rc = dpde_set_tuning(h, &best)) != DPDE_OK) break;
        enqueue_rebin(h, h->stream);
        if (cudaGetLastError() != cudaSuccess) { rc = fail(h, DPDE_ERR_CUDA, "rebinning the state"); break; }
        best.ms_per_step = best_ms;
    } while (false);
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    cudaStreamSynchronize(h->stream);
    cudaFree(save);
    if (rc == DPDE_OK && out) *out = best;
    return rc;
}

int dpde_step_launches(dpde_handle* h, int32_t scheme, int64_t* launches) {
    if (!h || !launches) return DPDE_ERR_ARG;
    if (scheme < DPDE_SER || scheme > DPDE_SSA) return fail(h, DPDE_ERR_ARG, "bad scheme");
    *launches = 0;
    if (h->N == 0) return DPDE_OK;
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    enqueue_step_any(h, h->cap_stream, 0.01, scheme);
    CK(h, cudaStreamEndCapture(h->cap_stream, &g));
    size_t nodes = 0;
    cudaError_t e = cudaGraphGetNodes(g, nullptr, &nodes);
    std::vector<cudaGraphNode_t> list(nodes);
    if (e == cudaSuccess && nodes > 0) e = cudaGraphGetNodes(g, list.data(), &nodes);
    int64_t kernels = 0;
    for (size_t k = 0; k < nodes && e == cudaSuccess; ++k) {
        cudaGraphNodeType type;
        e = cudaGraphNodeGetType(list[k], &type);
        if (e == cudaSuccess && type == cudaGraphNodeTypeKernel) ++kernels;
    }
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphGetNodes");
    *launches = kernels;
    return DPDE_OK;
}

int dpde_step_profiled(dpde_handle* h, int64_t n, double dt, int32_t scheme, double* phase_ms) {
    NvtxRange nvtx_range_("dpde_step_profiled");
    if (!h || !phase_ms) return DPDE_ERR_ARG;
    if (n < 0 || !(dt > 0) || !std::isfinite(dt) || scheme < DPDE_SER || scheme > DPDE_SSA)
        return fail(h, DPDE_ERR_ARG, "bad n, dt or scheme");
    if (h->N == 0) return dpde_step(h, n, dt, scheme, 0);
    for (auto& row : h->prof_ev)
        for (auto& ev : row)
            if (!ev) CK(h, cudaEventCreate(&ev));
    for (int64_t k = 0; k < n; ++k) {
        for (bool& u : h->prof_used) u = false;
        h->profiling = true;
        enqueue_step_any(h, h->stream, dt, scheme);
        h->profiling = false;
        CK(h, cudaGetLastError());
        CK(h, cudaStreamSynchronize(h->stream));
        for (int ph = 0; ph < DPDE_NUM_PHASES; ++ph) {
            if (!h->prof_used[ph]) continue;
            float ms = 0.f;
            CK(h, cudaEventElapsedTime(&ms, h->prof_ev[ph][0], h->prof_ev[ph][1]));
            phase_ms[ph] += ms;
        }
    }
    h->step += n;
    return DPDE_OK;
}

int dpde_sync(dpde_handle* h) {
    if (!h) return DPDE_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaGetLastError());
    return read_status(h);
}

int dpde_observables(dpde_handle* h, dpde_obs* out) {
    NvtxRange nvtx_range_("dpde_observables");
    if (!h || !out) return DPDE_ERR_ARG;
    if (h->mixed) enqueue_obs<float>(h, h->stream);
    else enqueue_obs<double>(h, h->stream);
    CK(h, cudaGetLastError());
    std::vector<double> host((size_t)NTERMS * h->R);
    CK(h, cudaMemcpyAsync(host.data(), h->obs_out, sizeof(double) * host.size(), cudaMemcpyDeviceToHost,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    bool neg = false, bad = false;
    for (int r = 0; r < h->R; ++r) {
        const double* t = host.data() + (size_t)NTERMS * r;
        const long long n = h->info[r].n;
        dpde_obs& o = out[r];
        o.K = t[0]; o.U = t[1]; o.Eint = t[2];
        o.E = o.U + o.K + o.Eint;
        o.P[0] = t[3]; o.P[1] = t[4]; o.P[2] = t[5];
        o.Tkin = n > 1 ? 2.0 * o.K / (3.0 * (double)(n - 1)) : 0.0;
        o.Tint = n > 0 ? (double)n / t[6] : 0.0;
        o.Tpot_num = t[7];
        o.Tpot_den = t[8];
        o.step = h->step;
        o.n = n;
        o.neg_eps = (int64_t)t[9];
        o.nonfinite = (int64_t)t[10];
        neg |= o.neg_eps > 0;
        bad |= o.nonfinite > 0;
    }
    int st = read_status(h);
    if (bad) return fail(h, DPDE_ERR_NONFINITE, "non-finite value in the state");
    if (neg) return fail(h, DPDE_ERR_NEG_EPS, "internal energy eps_i <= 0");
    return st;
}

namespace {
struct CkptHeader {
    uint64_t magic, N, R, precision, step, seed, cfg_hash, section_bytes;
};
uint64_t config_hash(const dpde_handle* h) {
    uint64_t x = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* b = (const unsigned char*)p;
        for (size_t i = 0; i < n; ++i) x = (x ^ b[i]) * 1099511628211ull;
    };
    mix(&h->prm, sizeof(h->prm));
    for (const dpde_replica& r : h->reps) mix(&r, sizeof(r));
    return x;
}
}  // namespace

int dpde_checkpoint(dpde_handle* h, void* buf, uint64_t* size) {
    NvtxRange nvtx_range_("dpde_checkpoint");
    if (!h || !size) return DPDE_ERR_ARG;
    const size_t N = (size_t)h->N;
    const size_t vsz = h->mixed ? sizeof(float4) : sizeof(d4);
    const size_t esz = h->mixed ? sizeof(ff) : sizeof(double);
    const size_t body = N * (3 * vsz + esz + sizeof(int));
    const size_t total = sizeof(CkptHeader) + body;
    if (!buf) {
        *size = total;
        return DPDE_OK;
    }
    if (*size < total) return fail(h, DPDE_ERR_ARG, "checkpoint buffer too small");
    CK(h, cudaStreamSynchronize(h->stream));
    CkptHeader hd{0x4450444543484b31ull, N, (uint64_t)h->R, (uint64_t)h->prm.precision, (uint64_t)h->step,
                  h->prm.seed, config_hash(h), body};
    unsigned char* out = (unsigned char*)buf;
    std::memcpy(out, &hd, sizeof(hd));
    out += sizeof(hd);
    const void* src[5] = {h->qA, h->pA, h->F, h->eA, h->cA};
    const size_t len[5] = {N * vsz, N * vsz, N * vsz, N * esz, N * sizeof(int)};
    for (int k = 0; k < 5; ++k) {
        if (len[k]) CK(h, cudaMemcpy(out, src[k], len[k], cudaMemcpyDeviceToHost));
        out += len[k];
    }
    *size = total;
    return DPDE_OK;
}

int dpde_restore(dpde_handle* h, const void* buf, uint64_t size) {
    NvtxRange nvtx_range_("dpde_restore");
    if (!h || !buf || size < sizeof(CkptHeader)) return DPDE_ERR_ARG;
    CkptHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    const size_t N = (size_t)h->N;
    const size_t vsz = h->mixed ? sizeof(float4) : sizeof(d4);
    const size_t esz = h->mixed ? sizeof(ff) : sizeof(double);
    const size_t body = N * (3 * vsz + esz + sizeof(int));
    if (hd.magic != 0x4450444543484b31ull || hd.N != N || hd.cfg_hash != config_hash(h) ||
        hd.section_bytes != body || size < sizeof(hd) + body)
        return fail(h, DPDE_ERR_ARG, "checkpoint does not match this handle");
    const unsigned char* in = (const unsigned char*)buf + sizeof(hd);
    void* dst[5] = {h->qA, h->pA, h->F, h->eA, h->cA};
    const size_t len[5] = {N * vsz, N * vsz, N * vsz, N * esz, N * sizeof(int)};
    CK(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 5; ++k) {
        if (len[k]) CK(h, cudaMemcpy(dst[k], in, len[k], cudaMemcpyHostToDevice));
        in += len[k];
    }
    long long s = (long long)hd.step;
    CK(h, cudaMemcpy(h->d_step, &s, sizeof(long long), cudaMemcpyHostToDevice));
    CK(h, cudaMemset(h->d_status, 0, sizeof(unsigned)));
    if (N > 0) enqueue_rebin(h, h->stream);
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(h->stream));
    h->step = s;
    return DPDE_OK;
}

int dpde_get_step(dpde_handle* h, int64_t* step) {
    if (!h || !step) return DPDE_ERR_ARG;
    *step = h->step;
    return DPDE_OK;
}

int dpde_destroy(dpde_handle* h) {
    if (!h) return DPDE_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return DPDE_OK;
}

const char* dpde_last_error(const dpde_handle* h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

int dpde_debug_philox(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
    if (n < 0 || (n > 0 && (!ctr || !key || !out))) return DPDE_ERR_ARG;
    if (n == 0) return DPDE_OK;
    uint4 *dc = nullptr, *dout = nullptr;
    uint2* dk = nullptr;
    cudaError_t e = cudaMalloc(&dc, 16 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dk, 8 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dout, 16 * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, 16 * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, 8 * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_debug_philox<<<ceil_div(n, 256), 256>>>((int)n, dc, dk, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, 16 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(dc); cudaFree(dk); cudaFree(dout);
    if (e != cudaSuccess) return fail(nullptr, DPDE_ERR_CUDA, cudaGetErrorString(e));
    return DPDE_OK;
}

int dpde_debug_gaussian(int64_t n, uint64_t seed, const uint32_t* step, const uint32_t* replica,
                        const uint32_t* id_a, const uint32_t* id_b, int32_t precision, double* out) {
    if (n < 0 || (n > 0 && (!step || !replica || !id_a || !id_b || !out))) return DPDE_ERR_ARG;
    if (n == 0) return DPDE_OK;
    uint32_t* d = nullptr;
    double* dout = nullptr;
    cudaError_t e = cudaMalloc(&d, 16 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dout, 24 * (size_t)n);
    const uint32_t* src[4] = {step, replica, id_a, id_b};
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        e = cudaMemcpy(d + (size_t)k * n, src[k], 4 * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const uint2 s = make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
        if (precision == DPDE_FP64)
            k_debug_gauss<double><<<ceil_div(n, 256), 256>>>((int)n, s, d, d + n, d + 2 * n, d + 3 * n, dout);
        else
            k_debug_gauss<float><<<ceil_div(n, 256), 256>>>((int)n, s, d, d + n, d + 2 * n, d + 3 * n, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, 24 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d); cudaFree(dout);
    if (e != cudaSuccess) return fail(nullptr, DPDE_ERR_CUDA, cudaGetErrorString(e));
    return DPDE_OK;
}

}  // extern "C"
