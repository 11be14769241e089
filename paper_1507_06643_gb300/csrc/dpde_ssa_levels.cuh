// dpde_ssa_levels.cuh -- the SSA sequence of every domain (Sec. III.A.2,
// III.B.2) executed by dependency levels, domain by domain, each domain's
// state held in shared memory.
//
// The SSA pair map of Eq. (SSA_ij) reads and writes the state of its two
// particles only, so two maps on disjoint particles commute exactly: the
// result of the sequence depends only on, for every particle, the order of
// the maps that touch it. Give map k of the sequence the level
//     lev(k) = 1 + max(lev of the last earlier map touching s_k,
//                      lev of the last earlier map touching t_k)
// (0 if none). Maps of one level touch disjoint particles, and running the
// levels in increasing order keeps, for every particle, the sequence order
// of its maps -- so the level-by-level execution is the sequence, bit for
// bit. At density 3 a domain of ~700 particles has ~3,600 maps in ~100
// levels (the per-class chains of the colour order are ~300 maps deep).
//
// Two kernels per step:
//   k_ssa_sched  one block per domain: stages the domain's forward entries
//                (partner slots, as the force pass wrote them) in shared
//                memory, walks the colour classes in order computing every
//                map's level (a thread per cell of the class: cells of one
//                class share no particle), then sorts the entries by level
//                into records (s, t, w) in global memory.
//   k_ssa_exec   one block per domain: stages (p, eps, id) of the domain,
//                then runs the levels in order, one thread per map, drawing
//                each pair's Gaussian on the fly (Philox is keyed on the ids),
//                with a block barrier between levels; writes the state back.
// Domains too large for the regular shared-memory capacities are deferred to
// a second launch of each kernel with ~2.5x larger capacities (several
// blocks per SM), and from there to a third with what ~200 KB hold; beyond
// those, the execution runs on the state in global memory (same levels, same
// bits), and a domain whose schedule does not fit at all is executed class by
// class along the colour order itself.
#pragma once

#include "dpde_kernels.cuh"

namespace dpde {

constexpr int SSA_MAXLEV = 1023;         // levels of one domain kept by the schedule
constexpr int SSA_LV_STRIDE = SSA_MAXLEV + 2;
constexpr int SCHED_THREADS = 128;
constexpr int SSA_LOAD_BATCH = 8;       // entries of a row taken together by the level walk
constexpr int SSA_COL_BATCH = 6;        // particles whose m-th entries a thread loads together
constexpr int SSA_EXEC_THREADS_MAX = 128;
constexpr int SSA_LOCAL_MAX = 65535;      // particles (and entries) of one domain: 16-bit local indices
constexpr int SSA_NLISTS = 5;             // deferred-domain lists of one step (see enqueue_ssa_levels)

// Domains of the SSA sequence: the cells of each domain sorted by colour
// class (`cells`), the NCOLOURS + 1 class starts of every domain in `cells`
// (`off`), and the first cell of every domain, then the total cell count
// (`cell0`). A domain is a contiguous cell (and slot) range.
struct SsaDomains {
    const int* cells;
    const int* off;
    const int* cell0;
    int n;
};

// The level schedule of every domain: per domain the record offsets of its
// levels (lv_off[d * SSA_LV_STRIDE + l], l = 0..nlev, records of level l in
// [lv_off[l], lv_off[l + 1])), its level count (lv_n[d]: nlev >= 0 from the
// regular launch, -3 - nlev from a deferred one, -1 no schedule (executed
// along the colour order), SSA_PENDING = -2 deferred and not yet scheduled),
// and the records, domain d's at [slot0(d) * cap, ...): (s_local | t_local
// << 16) and the weight w. The execution's regular launch, which may run
// beside the schedule's deferred launches, takes only lv_n >= -1, so it never
// reads a schedule that is still being written.
template <class T>
struct SsaLevels {
    int* lv_off;
    int* lv_n;
    uint32_t* rec_st;
    T* rec_w;
};

// shared bytes of k_ssa_sched for scap particles, ecap entries and ccap
// cells: cnt (16-bit counters of levels 0..SSA_MAXLEV + 1, two to a word) |
// cr[ccap] (the domain's cells in class order: local start | count << 16) |
// rowoff[scap + 1] | L[scap] | ent[ecap] (16-bit)
__host__ __device__ constexpr size_t ssa_sched_smem(int scap, int ecap, int ccap) {
    return (size_t)(SSA_LV_STRIDE / 2 + 1 + ccap) * sizeof(int) +
           (((size_t)(2 * scap + 1 + ecap) * 2 + 15) / 16) * 16;
}
// shared bytes of k_ssa_exec for scap staged particles: p | eps | id, after
// up to 31 bytes that align p to 32 bytes
template <class T>
__host__ __device__ constexpr size_t ssa_exec_smem(int scap) {
    return 32 + (size_t)scap * (sizeof(vec_t<T>) + sizeof(eps_t<T>) + sizeof(uint32_t));
}

// slot range [sb, se) of domain d
template <class T>
__device__ __forceinline__ void ssa_domain_range(const Ctx<T>& C, const SsaDomains& D, int d, int& sb, int& se) {
    sb = C.start[D.cell0[d]];
    se = C.start[D.cell0[d + 1]];
}

// Exclusive scan over n values v(i) held nowhere in particular: each thread
// takes a contiguous run; writes out[i] (16-bit) for i < n and returns the
// total. v is a callable.
template <class F>
__device__ __forceinline__ int block_scan_runs(int n, unsigned short* out, int* sh, F&& v) {
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int i0 = min(n, (int)threadIdx.x * per), i1 = min(n, i0 + per);
    int run = 0;
    for (int i = i0; i < i1; ++i) run += v(i);
    int total;
    int ex = block_exclusive_scan(run, sh, total);
    for (int i = i0; i < i1; ++i) {
        const int x = v(i);
        out[i] = (unsigned short)ex;
        ex += x;
    }
    return total;
}

// 16-bit level counters, two to a 32-bit word (a domain has at most
// SSA_LOCAL_MAX entries, so no count or offset reaches the upper half)
__device__ __forceinline__ int cnt_add(int* cnt, int l) {
    const int sh = (l & 1) << 4;
    return (atomicAdd(cnt + (l >> 1), 1 << sh) >> sh) & 0xffff;
}
__device__ __forceinline__ int cnt_get(const int* cnt, int l) { return (cnt[l >> 1] >> ((l & 1) << 4)) & 0xffff; }

// The forward entries of the domain's particles, entry index m outermost:
// a thread takes SSA_COL_BATCH particles i = i0 + tid + k blockDim (so a
// warp's lanes read consecutive words of each entry row [m N + i]) and, for
// every m below their row lengths, issues the loads of all of them before
// using them. use(i, e, v) gets the value load(i, m) of entry m of particle
// i, whose row starts at rowoff[i] (e = rowoff[i] + m).
template <class Load, class Use>
__device__ __forceinline__ void ssa_rows_mmajor(int nb, const unsigned short* rowoff, Load&& load, Use&& use) {
    const int bd = blockDim.x;
    for (int i0 = 0; i0 < nb; i0 += SSA_COL_BATCH * bd) {
        int e0[SSA_COL_BATCH], nf[SSA_COL_BATCH], mx = 0;
#pragma unroll
        for (int k = 0; k < SSA_COL_BATCH; ++k) {
            const int i = i0 + (int)threadIdx.x + k * bd;
            e0[k] = i < nb ? rowoff[i] : 0;
            nf[k] = i < nb ? rowoff[i + 1] - e0[k] : 0;
            mx = max(mx, nf[k]);
        }
        for (int m = 0; m < mx; ++m) {
            decltype(load(0, 0)) v[SSA_COL_BATCH];
#pragma unroll
            for (int k = 0; k < SSA_COL_BATCH; ++k)
                if (m < nf[k]) v[k] = load(i0 + (int)threadIdx.x + k * bd, m);
#pragma unroll
            for (int k = 0; k < SSA_COL_BATCH; ++k)
                if (m < nf[k]) use(i0 + (int)threadIdx.x + k * bd, e0[k] + m, v[k]);
        }
    }
}

// One domain's schedule on the calling block. Returns false (nothing written)
// when the domain exceeds scap particles, ecap entries or SSA_MAXLEV levels.
template <class T>
__device__ bool ssa_sched_domain(const Ctx<T>& C, const SsaDomains& D, const SsaLevels<T>& V, int d, int scap,
                                 int ecap, int ccap, bool deferred, unsigned char* smem) {
    __shared__ int sh[32];
    __shared__ int s_flag, s_nlev;
    __shared__ int s_off[NCOLOURS + 1];
    int sb, se;
    ssa_domain_range(C, D, d, sb, se);
    const int nb = se - sb;
    const int tid = threadIdx.x;
    if (nb > scap || nb > SSA_LOCAL_MAX) return false;
    int* cnt = reinterpret_cast<int*>(smem);
    unsigned int* cr = reinterpret_cast<unsigned int*>(cnt + SSA_LV_STRIDE / 2 + 1);
    unsigned short* rowoff = reinterpret_cast<unsigned short*>(cr + ccap);
    unsigned short* L = rowoff + scap + 1;
    unsigned short* ent = L + scap;    // partner (local slot) of each entry, then its level
    if (tid == 0) {
        s_flag = 0;
        s_nlev = 0;
    }
    for (int l = tid; l <= SSA_LV_STRIDE / 2; l += blockDim.x) cnt[l] = 0;
    const int* off = D.off + (size_t)d * (NCOLOURS + 1);
    for (int k = tid; k <= NCOLOURS; k += blockDim.x) s_off[k] = __ldg(off + k);
    __syncthreads();
    // the domain's cells in class order, start and particle count, read once
    // here rather than class by class in the walk (a domain with more cells
    // than ccap reads them in the walk)
    const int cbase = s_off[0], ncell = s_off[NCOLOURS] - cbase;
    const bool cstaged = ncell <= ccap;
    if (cstaged)
        for (int u = tid; u < ncell; u += blockDim.x) {
            const int c = __ldg(D.cells + cbase + u);
            const int a = C.start[c], b = C.start[c + 1];
            cr[u] = (unsigned int)(a - sb) | ((unsigned int)(b - a) << 16);
        }
    // 1. row offsets of the domain's forward entries (16-bit: checked below)
    const int* fwd_n = C.fwd_n + sb;
    const int E = block_scan_runs(nb, rowoff, sh, [&](int i) { return fwd_n[i]; });
    if (E > ecap || E > SSA_LOCAL_MAX) return false;   // uniform over the block
    if (tid == 0) rowoff[nb] = (unsigned short)E;
    for (int i = tid; i < nb; i += blockDim.x) L[i] = 0;
    __syncthreads();   // the rows' offsets were written by other threads
    const size_t N = (size_t)C.N;
    const int* fj = C.fwd_j + sb;   // entry m of local particle i at fj[m N + i]
    const T* fw = C.fwd_w + sb;
    // 2. partner slots, local
    ssa_rows_mmajor(
        nb, rowoff, [&](int i, int m) { return __ldg(fj + (size_t)m * N + i) - sb; },
        [&](int, int e, int t) {
            if ((unsigned)t >= (unsigned)nb) s_flag = 1;   // never by construction
            ent[e] = (unsigned short)min(max(t, 0), nb - 1);
        });
    __syncthreads();
    if (s_flag) {
        if (tid == 0) flag(C.status, ST_DOMAIN);
        return false;
    }
    // 3. levels, class by class. Eight lanes take one cell of the class (the
    //    cells of a class share no particle) and walk its rows -- the cell's
    //    particles in slot order -- a chunk of up to eight entries at a time:
    //    the partners of a row are distinct particles, so their levels are
    //    loaded at once, and within the chunk the levels follow from a
    //    prefix maximum across the lanes,
    //      lev_j = j + 1 + max(L_s, max_{k <= j} (L[t_k] - k)),
    //    which is the recurrence lev_j = 1 + max(lev_{j-1}, L[t_j]) unrolled.
    const int lane = tid & 31, sub = lane & 7, gbase = lane & ~7;
    const int group = tid >> 3, ngroups = blockDim.x >> 3;
    int mylev = 0;
    for (int k = 0; k < NCOLOURS; ++k) {
        const int k0 = s_off[k], k1 = s_off[k + 1];
        if (k1 == k0) continue;   // uniform over the block
        for (int u0 = k0; u0 < k1; u0 += ngroups) {   // uniform over the block
            const int u = u0 + group;
            int s0 = 0, nrow = 0;
            if (u < k1) {
                if (cstaged) {
                    const unsigned int v = cr[u - cbase];
                    s0 = (int)(v & 0xffffu);
                    nrow = (int)(v >> 16);
                } else {
                    const int c = __ldg(D.cells + u);
                    s0 = C.start[c] - sb;
                    nrow = C.start[c + 1] - sb - s0;
                }
            }
            const int wrows = __reduce_max_sync(0xffffffffu, nrow);
            for (int r = 0; r < wrows; ++r) {
                const bool ract = r < nrow;
                const int i = s0 + r;
                int Ls = ract ? L[i] : 0;
                const int e0 = ract ? rowoff[i] : 0, n = ract ? rowoff[i + 1] - e0 : 0;
                const int wchunks = __reduce_max_sync(0xffffffffu, (n + 7) >> 3);
                for (int ch = 0; ch < wchunks; ++ch) {
                    const int j = (ch << 3) + sub;   // entry of the row
                    const bool ea = j < n;
                    const int t = ea ? ent[e0 + j] : 0;
                    int a = ea ? (int)L[t] - sub : -65536;
#pragma unroll
                    for (int o = 1; o < 8; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, a, o, 8);
                        if (sub >= o) a = max(a, y);
                    }
                    const int lv = min(max(Ls, a) + sub + 1, 65535);
                    if (ea) {
                        L[t] = (unsigned short)lv;
                        ent[e0 + j] = (unsigned short)lv;
                    }
                    const int last = min(n - (ch << 3), 8) - 1;   // last entry of this chunk
                    const int lvl = __shfl_sync(0xffffffffu, lv, gbase + max(last, 0));
                    if (last >= 0) Ls = lvl;
                }
                if (ract) {
                    if (sub == 0) L[i] = (unsigned short)Ls;
                    mylev = max(mylev, Ls);
                }
                __syncwarp();   // the row's level writes, before the next row reads them
            }
        }
        __syncthreads();
    }
    atomicMax(&s_nlev, mylev);
    __syncthreads();
    const int nlev = s_nlev;
    if (nlev > SSA_MAXLEV) return false;
    // 4. records sorted by level: counts, offsets, scatter
    for (int e = tid; e < E; e += blockDim.x) cnt_add(cnt, ent[e]);
    __syncthreads();
    int* lvo = V.lv_off + (size_t)d * SSA_LV_STRIDE;
    if (tid < 32) {
        // exclusive scan of the counts of levels 1..nlev: lvo[l - 1] = start
        // of level l, lvo[nlev] = E; the counters become the cursors
        int carry = 0;
        for (int l0 = 1; l0 <= nlev + 1; l0 += 32) {
            const int l = l0 + tid;
            const int v = l <= nlev ? cnt_get(cnt, l) : 0;
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (tid >= o) x += y;
            }
            if (l <= nlev + 1) lvo[l - 1] = carry + x - v;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
    }
    __syncthreads();
    for (int l = tid; l <= SSA_LV_STRIDE / 2; l += blockDim.x) {
        // cursor pair (2l, 2l + 1) = level starts (lvo[2l - 1], lvo[2l])
        const int lo = 2 * l >= 1 && 2 * l <= nlev ? lvo[2 * l - 1] : 0;
        const int hi = 2 * l + 1 <= nlev ? lvo[2 * l] : 0;
        cnt[l] = lo | (hi << 16);
    }
    __syncthreads();
    // the partners again from the force pass's list (just read: cached), the
    // weights with them
    const size_t base = (size_t)sb * C.nbr_cap;
    struct TW {
        int t;
        T w;
    };
    ssa_rows_mmajor(
        nb, rowoff,
        [&](int i, int m) {
            const size_t at = (size_t)m * N + i;
            return TW{__ldg(fj + at) - sb, __ldg(fw + at)};
        },
        [&](int i, int e, const TW& x) {
            const int pos = cnt_add(cnt, ent[e]);
            V.rec_st[base + pos] = (uint32_t)i | ((uint32_t)min(max(x.t, 0), nb - 1) << 16);
            V.rec_w[base + pos] = x.w;
        });
    if (tid == 0) V.lv_n[d] = deferred ? -3 - nlev : nlev;
    return true;
}

// level count of a schedule stored as lv_n (see SsaLevels); -1 without one
__device__ __forceinline__ int ssa_nlev(int v) { return v <= -3 ? -3 - v : v; }

// One launch over the domains. Regular form (list == nullptr): block u takes
// domain d0 + u. Deferred form: the blocks loop over `list`. A domain beyond
// the launch's capacities is passed on to `defer` when one is given (lv_n =
// SSA_PENDING until a later launch schedules it), else left without a
// schedule (lv_n = -1: executed along the colour order).
constexpr int SSA_PENDING = -2;

template <class T>
__global__ void __launch_bounds__(SCHED_THREADS, 8) k_ssa_sched(Ctx<T> C, SsaDomains D, SsaLevels<T> V, int scap,
                                                                 int ecap, int ccap, int d0,
                                                                 const int* __restrict__ list,
                                                                 const int* __restrict__ nlist, int* defer,
                                                                 int* ndefer) {
    extern __shared__ __align__(16) unsigned char sched_smem[];
    const int n = list ? *nlist : (int)gridDim.x;
    for (int u = blockIdx.x; u < n; u += gridDim.x) {
        const int d = list ? list[u] : d0 + u;
        if (!ssa_sched_domain(C, D, V, d, scap, ecap, ccap, list != nullptr, sched_smem) && threadIdx.x == 0) {
            V.lv_n[d] = defer ? SSA_PENDING : -1;
            if (defer) defer[atomicAdd(ndefer, 1)] = d;
        }
        __syncthreads();
    }
}

// The levels of domain d on the state (P, Es, ID), indexed by local slot.
// A thread's first map of every level (its "pass 0") runs in a three-stage
// software pipeline: the record of level l + 2 is loaded, the Gaussian of
// level l + 1 drawn, and the map of level l applied in the same iteration, so
// neither the record's global-memory latency nor the Philox rounds sit between
// two level barriers. Further maps of a crowded level follow unpipelined.
template <class T>
__device__ __forceinline__ void ssa_exec_levels(const Ctx<T>& C, const SsaLevels<T>& V, int d, int sb, int rep,
                                                vec_t<T>* P, eps_t<T>* Es, const uint32_t* ID, T dt,
                                                T sqrt_dt) {
    const RepInfo& R = C.reps[rep];
    const T amp0 = T(2) * C.sigma * sqrt_dt;   // amplitude of the map as gamma -> 0
    const T k2 = T(2) * dt * C.inv_m;
    const uint32_t step = (uint32_t)*C.step;
    const int nlev = ssa_nlev(V.lv_n[d]);
    const int* lvo = V.lv_off + (size_t)d * SSA_LV_STRIDE;
    const size_t base = (size_t)sb * C.nbr_cap;
    const uint32_t* rst = V.rec_st + base;
    const T* rw = V.rec_w + base;
    const int tid = threadIdx.x;
    auto apply = [&](uint32_t st, const vec_t<T>& g) {
        const int s = (int)(st & 0xffffu), t = (int)(st >> 16);
        vec_t<T> ps = P[s];
        eps_t<T> es = Es[s];
        T bs = ps.w;
        vec_t<T> pt = P[t];
        eps_t<T> et = Es[t];
        ssa_pair_map(C, R, ps, es, bs, pt, et, g, k2, amp0);
        ps.w = bs;
        P[s] = ps;
        Es[s] = es;
        P[t] = pt;
        Es[t] = et;
    };
    auto gauss = [&](uint32_t st, T w) {
        const T3<T> G = pair_gauss<T>(C.seed, step, (uint32_t)rep, ID[st & 0xffffu], ID[st >> 16]);
        vec_t<T> g;
        g.x = G.x;
        g.y = G.y;
        g.z = G.z;
        g.w = w;
        return g;
    };
    // level starts o[l] for l = 0..nlev, read three levels ahead
    auto lv_start = [&](int l) { return l <= nlev ? __ldg(lvo + l) : 0; };
    int o0 = lv_start(0), o1 = lv_start(1), o2 = lv_start(2), o3 = lv_start(3);
    // pass-0 records of levels 0 and 1
    bool v0 = 0 < nlev && o0 + tid < o1, v1 = 1 < nlev && o1 + tid < o2;
    uint32_t st0 = v0 ? __ldg(rst + o0 + tid) : 0u, st1 = v1 ? __ldg(rst + o1 + tid) : 0u;
    T w0 = v0 ? __ldg(rw + o0 + tid) : T(0), w1 = v1 ? __ldg(rw + o1 + tid) : T(0);
    vec_t<T> g0{};
    if (v0) g0 = gauss(st0, w0);
    for (int l = 0; l < nlev; ++l) {
        // record of level l + 2
        const bool v2 = l + 2 < nlev && o2 + tid < o3;
        const uint32_t st2 = v2 ? __ldg(rst + o2 + tid) : 0u;
        const T w2 = v2 ? __ldg(rw + o2 + tid) : T(0);
        const int o4 = lv_start(l + 4);
        // Gaussian of level l + 1 (a warp without a map there skips it), then
        // the map of level l
        vec_t<T> g1{};
        if (v1) g1 = gauss(st1, w1);
        if (v0) apply(st0, g0);
        for (int r = o0 + tid + blockDim.x; r < o1; r += blockDim.x) {
            const uint32_t st = __ldg(rst + r);
            apply(st, gauss(st, __ldg(rw + r)));
        }
        __syncthreads();
        o0 = o1; o1 = o2; o2 = o3; o3 = o4;
        v0 = v1; st0 = st1; g0 = g1;
        v1 = v2; st1 = st2; w1 = w2;
    }
}

// Domain d without a schedule: its colour classes in order on the state in
// global memory, a thread per cell of the class (the colour order itself).
template <class T>
__device__ void ssa_exec_classes(const Ctx<T>& C, const SsaDomains& D, int d, int rep, T dt, T sqrt_dt) {
    const RepInfo& R = C.reps[rep];
    const T amp0 = T(2) * C.sigma * sqrt_dt;
    const T k2 = T(2) * dt * C.inv_m;
    const uint32_t step = (uint32_t)*C.step;
    const size_t N = (size_t)C.N;
    const int* off = D.off + (size_t)d * (NCOLOURS + 1);
    for (int k = 0; k < NCOLOURS; ++k) {
        const int k0 = off[k], k1 = off[k + 1];
        if (k1 == k0) continue;
        for (int u = k0 + threadIdx.x; u < k1; u += blockDim.x) {
            const int c = D.cells[u];
            for (int s = C.start[c]; s < C.start[c + 1]; ++s) {
                const int nf = C.fwd_n[s];
                if (nf == 0) continue;
                vec_t<T> ps = C.pB[s];
                eps_t<T> es = C.eB[s];
                T bs = ps.w;
                const uint32_t ids = C.idB[s];
                for (int m = 0; m < nf; ++m) {
                    const int t = C.fwd_j[(size_t)m * N + s];
                    const T3<T> G = pair_gauss<T>(C.seed, step, (uint32_t)rep, ids, C.idB[t]);
                    vec_t<T> g;
                    g.x = G.x;
                    g.y = G.y;
                    g.z = G.z;
                    g.w = C.fwd_w[(size_t)m * N + s];
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
        __syncthreads();
    }
}

// One domain on the calling block: staged in shared memory when it fits in
// scap slots, else deferred (defer given) or run on global memory (defer ==
// nullptr). The regular launch skips a domain whose schedule was deferred.
template <class T>
__device__ void ssa_exec_domain(const Ctx<T>& C, const SsaDomains& D, const SsaLevels<T>& V, int d, int scap,
                                bool regular, int* defer, int* ndefer, T dt, T sqrt_dt, unsigned char* smem) {
    int sb, se;
    ssa_domain_range(C, D, d, sb, se);
    const int nb = se - sb;
    if (nb == 0) return;
    const int v = V.lv_n[d];
    const int rep = C.rep_of_cell[D.cell0[d]];
    // deferred by the regular schedule: scheduled and executed by the deferred
    // launches (perhaps running beside this one)
    if (regular && v <= SSA_PENDING) return;
    const int nlev = ssa_nlev(v);
    if (nlev < 0) {   // no schedule, even with the largest capacities: the colour order itself
        ssa_exec_classes(C, D, d, rep, dt, sqrt_dt);
        return;
    }
    if (nb > scap) {
        if (defer) {
            if (threadIdx.x == 0) defer[atomicAdd(ndefer, 1)] = d;
            return;
        }
        ssa_exec_levels(C, V, d, sb, rep, C.pB + sb, C.eB + sb, C.idB + sb, dt, sqrt_dt);
        return;
    }
    vec_t<T>* P = reinterpret_cast<vec_t<T>*>(((size_t)smem + 31) & ~(size_t)31);
    eps_t<T>* Es = reinterpret_cast<eps_t<T>*>(P + scap);
    uint32_t* ID = reinterpret_cast<uint32_t*>(Es + scap);
    // four particles per thread in flight
    for (int i0 = threadIdx.x; i0 < nb; i0 += 4 * blockDim.x) {
        vec_t<T> pv[4];
        eps_t<T> ev[4];
        uint32_t iv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * (int)blockDim.x;
            if (i < nb) {
                pv[u] = C.pB[sb + i];
                ev[u] = C.eB[sb + i];
                iv[u] = C.idB[sb + i];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * (int)blockDim.x;
            if (i < nb) {
                P[i] = pv[u];
                Es[i] = ev[u];
                ID[i] = iv[u];
            }
        }
    }
    __syncthreads();
    ssa_exec_levels(C, V, d, sb, rep, P, Es, ID, dt, sqrt_dt);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        C.pB[sb + i] = P[i];
        C.eB[sb + i] = Es[i];
    }
}

// Regular form (list == nullptr): block u takes domain d0 + u, leaving out
// the domains the regular schedule deferred (the deferred launches execute
// them). Deferred form: the blocks loop over `list`. A domain with more than
// scap particles is passed on to `defer` when one is given, else run on the
// state in global memory.
template <class T>
__global__ void __launch_bounds__(SSA_EXEC_THREADS_MAX) k_ssa_exec(Ctx<T> C, SsaDomains D, SsaLevels<T> V,
                                                                    int scap, int d0, const int* __restrict__ list,
                                                                    const int* __restrict__ nlist, int* defer,
                                                                    int* ndefer, T dt, T sqrt_dt) {
    extern __shared__ __align__(16) unsigned char exec_smem[];
    const int n = list ? *nlist : (int)gridDim.x;
    for (int u = blockIdx.x; u < n; u += gridDim.x) {
        ssa_exec_domain(C, D, V, list ? list[u] : d0 + u, scap, list == nullptr, defer, ndefer, dt, sqrt_dt,
                        exec_smem);
        __syncthreads();
    }
}

}  // namespace dpde
