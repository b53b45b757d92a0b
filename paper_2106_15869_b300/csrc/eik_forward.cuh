// eik_forward.cuh -- forward kernels of the improved fast iterative method
// (Algorithm 2, Sec. 3.1.2) at tile granularity, for sm_103a.
//
// A tile of BX x BY x BZ nodes is the unit of the Active and Remedy sets.
// One warp owns one tile at a time: each lane holds NPL = V/32 nodes (node
// q = lane + 32 m, so loads and stores of the brick are coalesced), the warp
// stages the tile plus a one-node halo of phi in its own slice of shared
// memory, keeps tau in registers, and relaxes phi <- min(phi, eq.(6) root) in
// place until a sweep changes nothing (warp ballot).  Warps fetch tiles from
// the current list independently (one atomic per tile, prefetched one visit
// ahead), so there is no CTA-wide barrier on the tile path and each SM keeps
// dozens of tiles in flight.
//
// Step 1 (k_init, k_sources): phi = +inf, tau = h/F, sources fixed, Active =
//   the tiles holding the sources' neighbours.
// Step 2 (update_pass): an Active tile whose visit changes nothing joins
//   Source and activates its Distant face-neighbour tiles (no convergence check
//   of neighbours); a tile that changed stays Active.
// Step 3 (detect_pass, remedy_pass): one recomputation over all tiles seeds
//   Remedy with the tiles holding a node whose root is below its value; a
//   Remedy tile is relaxed (decrease only) and lists the neighbour tiles across
//   the faces where its values dropped.  Both loops run until their list is
//   empty.
#pragma once

#include <cstddef>

#include "eik_common.cuh"

namespace eik {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerCta = 8;

template <class T>
struct FwdParams {
    const InstDesc *desc;
    int B;
    int n_tiles;                 // total tiles over all instances
    int *tile_inst;
    int *tile_nb;                // [n_tiles][6] neighbour tile ids (-1 outside)
    int *tstate;
    int *tstamp;
    unsigned *tkey;              // [2][n_tiles] encoded list keys (ordered schedule)
    float *inst_scale;           // [B] 1/delta of each instance (ordered schedule)
    double *inst_acc;            // [B][2] sum of F and count of F > 0 (for delta)
    int ordered;                 // 1 = bucketed order of the lists
    float order;                 // bucket width in tile-crossing times
    int *list0, *list1;
    T *phi_t, *tau_t;
    Ctl *ctl;
    long long max_iters;
    int skip_remedy;
    int max_sweeps;              // cap on in-tile sweeps per visit
    const T *F;                  // packed input speeds
    const long long *src_idx;
    const T *src_val;
    long long n_src;
    T *phi_out;                  // packed output
};

template <int BX, int BY, int BZ>
struct TileGeom {
    static constexpr int V = BX * BY * BZ;
    static constexpr int NPL = V / 32;                      // nodes per lane
    static constexpr int SX = BX + 2, SY = BY + 2, SZ = BZ + 2;
    static constexpr int S = SX * SY * SZ;                  // staged values per warp
    static constexpr int FX = BY * BZ, FY = BX * BZ, FZ = BX * BY;
    static constexpr int HALO = 2 * (FX + FY + FZ);
    // staged halo values per visit: a 2D tile (BZ == 1) of a 2D grid never has
    // z neighbours, so its z planes stay +inf from init_stage()
    static constexpr int HALO_LOADED = BZ == 1 ? 2 * (FX + FY) : HALO;
    static_assert(V % 32 == 0, "tile volume must be a multiple of 32");
    static __device__ __forceinline__ int sidx(int x, int y, int z) { return ((z + 1) * SY + (y + 1)) * SX + (x + 1); }
    static __device__ __forceinline__ int sidx_of(int q) { return sidx(q % BX, (q / BX) % BY, q / (BX * BY)); }
    static __device__ __forceinline__ int faces_of(int q) {
        const int x = q % BX, y = (q / BX) % BY, z = q / (BX * BY);
        return (x == 0 ? 1 : 0) | (x == BX - 1 ? 2 : 0) | (y == 0 ? 4 : 0) | (y == BY - 1 ? 8 : 0) |
               (z == 0 ? 16 : 0) | (z == BZ - 1 ? 32 : 0);
    }
    // halo element h: face f, its slot in the staged block, and the node of
    // the neighbour tile across f that it copies
    static __device__ __forceinline__ void halo_of(int h, int &f, int &slot, int &src) {
        int a, b, r = h;
        if (r < 2 * FX) { f = r / FX; r %= FX; a = r % BY; b = r / BY; }
        else if ((r -= 2 * FX) < 2 * FY) { f = 2 + r / FY; r %= FY; a = r % BX; b = r / BX; }
        else { r -= 2 * FY; f = 4 + r / FZ; r %= FZ; a = r % BX; b = r / BX; }
        switch (f) {
            case 0: slot = sidx(-1, a, b); src = (b * BY + a) * BX + (BX - 1); break;
            case 1: slot = sidx(BX, a, b); src = (b * BY + a) * BX; break;
            case 2: slot = sidx(a, -1, b); src = (b * BY + (BY - 1)) * BX + a; break;
            case 3: slot = sidx(a, BY, b); src = (b * BY) * BX + a; break;
            case 4: slot = sidx(a, b, -1); src = ((BZ - 1) * BY + b) * BX + a; break;
            default: slot = sidx(a, b, BZ); src = (b * BX) + a; break;
        }
    }
};

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_in_cta() { return threadIdx.x >> 5; }

// Warp-aggregated list append: every lane with `want` appends its `g`; with a
// key array, the leader also lowers *kmin to the smallest key appended.
__device__ __forceinline__ void warp_push(Ctl *ctl, int *cnt, int *list, int cap, bool want, int g,
                                          unsigned *kmin = nullptr, unsigned key = 0xffffffffu) {
    const unsigned m = __ballot_sync(kFull, want);
    if (!m) return;
    const int lane = lane_id();
    const int leader = __ffs(m) - 1;
    int base = 0;
    unsigned kk = 0xffffffffu;
    if (kmin) kk = __reduce_min_sync(kFull, want ? key : 0xffffffffu);
    if (lane == leader) {
        base = atomicAdd(cnt, __popc(m));
        if (kmin) atomicMin(kmin, kk);
    }
    base = __shfl_sync(kFull, base, leader);
    if (want) {
        const int pos = base + __popc(m & ((1u << lane) - 1));
        if (pos < cap) __stcg(list + pos, g);
        else atomicOr(&ctl->flags, kFlagOverflow);
    }
}

// Fill a warp's staged block with +inf once per launch (the z planes of a 2D
// tile are never loaded afterwards).
template <class T, int BX, int BY, int BZ>
__device__ __forceinline__ void init_stage(T *sm) {
    for (int q = lane_id(); q < TileGeom<BX, BY, BZ>::S; q += 32) sm[q] = Num<T>::inf();
    __syncwarp();
}

// One visit's staged tile: load interior (registers + smem) and halo.
template <class T, int BX, int BY, int BZ>
__device__ __forceinline__ void stage_tile(const FwdParams<T> &P, T *sm, int g, int nbf,
                                           T (&v)[TileGeom<BX, BY, BZ>::NPL], T (&tau)[TileGeom<BX, BY, BZ>::NPL]) {
    using G = TileGeom<BX, BY, BZ>;
    const int lane = lane_id();
    const T *pg = P.phi_t + (size_t)g * G::V;
    const T *tg = P.tau_t + (size_t)g * G::V;
#pragma unroll
    for (int m = 0; m < G::NPL; ++m) {
        v[m] = __ldcg(pg + lane + 32 * m);
        tau[m] = __ldcg(tg + lane + 32 * m);
    }
#pragma unroll
    for (int m = 0; m < G::NPL; ++m) sm[G::sidx_of(lane + 32 * m)] = v[m];
#pragma unroll
    for (int m = 0; m < (G::HALO_LOADED + 31) / 32; ++m) {
        const int h = lane + 32 * m;
        int f = 0, slot = 0, src = 0;
        if (h < G::HALO_LOADED) G::halo_of(h, f, slot, src);
        const int n = __shfl_sync(kFull, nbf, f);
        if (h < G::HALO_LOADED) {
            T hv = Num<T>::inf();
            if (n >= 0) hv = __ldcg(P.phi_t + (size_t)n * G::V + src);
            sm[slot] = hv;
        }
    }
    __syncwarp();
}

// Slots (m) whose nodes neighbour a node of a slot in M.  Node q = lane + 32 m:
// x neighbours share the slot (BX divides 32), y neighbours are in m or m +- 1,
// z neighbours in m +- max(1, BX*BY/32).
template <int BX, int BY, int BZ>
__device__ __forceinline__ unsigned spread_slots(unsigned M) {
    constexpr int NPL = TileGeom<BX, BY, BZ>::NPL;
    constexpr int DZ = (BX * BY) / 32 > 0 ? (BX * BY) / 32 : 1;
    static_assert(32 % BX == 0, "a tile row must not straddle a 32-node slot");
    const unsigned a = M | (M << 1) | (M >> 1) | (M << DZ) | (M >> DZ);
    return NPL >= 32 ? a : (a & ((1u << NPL) - 1u));
}

// In-place relaxation of the staged tile until a sweep changes nothing (or the
// sweep cap).  The first sweep recomputes every node; later sweeps recompute
// only the slots next to a slot that changed in the previous sweep (a node
// whose neighbours did not change cannot change), which the warp decides
// uniformly from a ballot.  Returns the sweep count; `mine` = bit m set when
// node m of this lane dropped; `first_changed` = the first sweep changed some
// node.
template <class T, int BX, int BY, int BZ>
__device__ __forceinline__ int relax_tile(T *sm, T (&v)[TileGeom<BX, BY, BZ>::NPL],
                                          const T (&tau)[TileGeom<BX, BY, BZ>::NPL], int max_sweeps,
                                          unsigned &mine, bool &first_changed) {
    using G = TileGeom<BX, BY, BZ>;
    const int lane = lane_id();
    mine = 0;
    first_changed = false;
    unsigned act = G::NPL >= 32 ? ~0u : ((1u << G::NPL) - 1u);
    int s = 0;
    for (;;) {
        unsigned ch = 0;
#pragma unroll
        for (int m = 0; m < G::NPL; ++m) {
            if ((act >> m & 1) && !(tau[m] < T(0))) {
                const int c = G::sidx_of(lane + 32 * m);
                const T ax = vmin(sm[c - 1], sm[c + 1]);
                const T ay = vmin(sm[c - G::SX], sm[c + G::SX]);
                const T az = vmin(sm[c - G::SX * G::SY], sm[c + G::SX * G::SY]);
                const T u = local_solve<T>(ax, ay, az, tau[m]);
                if (u < v[m]) { v[m] = u; sm[c] = u; ch |= 1u << m; }
            }
        }
        mine |= ch;
        ++s;
        __syncwarp();
        const unsigned M = __reduce_or_sync(kFull, ch);
        if (s == 1) first_changed = M != 0;
        if (!M || s >= max_sweeps) break;
        act = spread_slots<BX, BY, BZ>(M);
    }
    return s;
}

// faces (bit f) holding a node that dropped in this visit, over the warp
template <int BX, int BY, int BZ>
__device__ __forceinline__ int changed_faces(unsigned mine) {
    using G = TileGeom<BX, BY, BZ>;
    int f = 0;
#pragma unroll
    for (int m = 0; m < G::NPL; ++m)
        if (mine >> m & 1) f |= G::faces_of(lane_id() + 32 * m);
    return (int)__reduce_or_sync(kFull, (unsigned)f);
}

template <class T, int BX, int BY, int BZ>
__device__ __forceinline__ void write_back(const FwdParams<T> &P, int g, unsigned mine,
                                           const T (&v)[TileGeom<BX, BY, BZ>::NPL]) {
    using G = TileGeom<BX, BY, BZ>;
    T *pg = P.phi_t + (size_t)g * G::V;
#pragma unroll
    for (int m = 0; m < G::NPL; ++m)
        if (mine >> m & 1) __stcg(pg + lane_id() + 32 * m, v[m]);
}

// Static assignment of list entries: warp w of the launch takes entries
// w, w + W, w + 2W, ... (W = warps in the launch); no atomics on the fetch path.
__device__ __forceinline__ int warp_global() { return blockIdx.x * kWarpsPerCta + warp_in_cta(); }
__device__ __forceinline__ int warps_total() { return gridDim.x * kWarpsPerCta; }

// ---------------------------------------------------------------- ordering
// Optional bucketed order of the tile lists (the "order" option).  Every
// listed tile carries a key: a lower bound of the values that can still
// reach it (the smallest incoming face value, or its own value), scaled by
// 1/delta of its instance, delta = order * (tile edge) * h / mean(F), i.e.
// `order` tile-crossing times.  An iteration visits the listed tiles whose
// key lies within one bucket of the smallest key in the list and defers the
// others to the next list unvisited.  The sets and their rules are those of
// Algorithm 2; only the iteration in which a listed tile is visited changes,
// and the fixed point reached does not depend on that (the discrete solution
// is unique).  Keys live in two parities: pushes for iteration it+1 write
// tkey[(it+1)&1], the visit in iteration it reads and clears tkey[it&1].
struct OrderCtx {
    bool on;
    unsigned kmin;      // smallest key listed for this iteration (encoded)
    float theta;        // visit iff key < theta (or every key is +inf)
};

__device__ __forceinline__ OrderCtx order_begin(bool on, unsigned kmin) {
    OrderCtx o;
    o.on = on;
    o.kmin = on ? kmin : kKeyInf;
    o.theta = key_dec(o.kmin) + 1.0f;
    return o;
}

__device__ __forceinline__ bool order_visit(const OrderCtx &o, unsigned key) {
    return !o.on || o.kmin == kKeyInf || key_dec(key) < o.theta;
}

// warp min of one float per lane, encoded
__device__ __forceinline__ unsigned warp_min_key(float k) { return __reduce_min_sync(kFull, key_enc(k)); }

// per-face minimum over this lane's nodes selected by `sel`, for face f
template <class T, int BX, int BY, int BZ>
__device__ __forceinline__ float face_min(unsigned sel, const T (&v)[TileGeom<BX, BY, BZ>::NPL], int f) {
    using G = TileGeom<BX, BY, BZ>;
    float m = __int_as_float(0x7f800000);
#pragma unroll
    for (int q = 0; q < G::NPL; ++q)
        if ((sel >> q & 1) && (G::faces_of(lane_id() + 32 * q) >> f & 1)) m = fminf(m, (float)v[q]);
    return m;
}

// ---------------------------------------------------------------- Step 2
// One pass over the Active list of iteration `it` (slot it % 3).
template <class T, int BX, int BY, int BZ>
__device__ void update_pass(const FwdParams<T> &P, T *sm, int it, int n, unsigned kmin_cur, long long &st_tiles,
                            long long &st_sweeps, long long &st_def) {
    using G = TileGeom<BX, BY, BZ>;
    Ctl *ctl = P.ctl;
    const int nslot = (it + 1) % 3;
    const int *in = (it & 1) ? P.list1 : P.list0;
    int *out = (it & 1) ? P.list0 : P.list1;
    unsigned *kcur = P.tkey + (size_t)(it & 1) * P.n_tiles;
    unsigned *knext = P.tkey + (size_t)((it + 1) & 1) * P.n_tiles;
    const int lane = lane_id();
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // slot (it+2)%3 was last read in iteration it-1
        ctl->cnt[(it + 2) % 3] = 0;
        ctl->kmin[(it + 2) % 3] = kKeyInf;
    }
    const OrderCtx ord = order_begin(P.ordered, kmin_cur);
    n = min(n, P.n_tiles);                       // n > n_tiles only after an overflow
    for (int idx = warp_global(); idx < n; idx += warps_total()) {
        const int g = __ldcg(in + idx);
        unsigned key = kKeyInf;
        if (ord.on) {
            if (lane == 0) key = atomicExch(kcur + g, kKeyInf);
            key = __shfl_sync(kFull, key, 0);
            if (!order_visit(ord, key)) {        // deferred: listed again, not visited
                if (lane == 0) {
                    atomicMin(knext + g, key);
                    st_def++;
                }
                warp_push(ctl, &ctl->cnt[nslot], out, P.n_tiles, lane == 0, g, &ctl->kmin[nslot], key);
                continue;
            }
        }
        const int nbf = lane < 6 ? __ldcg(P.tile_nb + 6 * g + lane) : -1;
        T v[G::NPL], tau[G::NPL];
        stage_tile<T, BX, BY, BZ>(P, sm, g, nbf, v, tau);
        unsigned mine;
        bool changed;
        const int s = relax_tile<T, BX, BY, BZ>(sm, v, tau, P.max_sweeps, mine, changed);
        write_back<T, BX, BY, BZ>(P, g, mine, v);
        if (lane == 0) { st_tiles++; st_sweeps += s; }
        if (changed) {
            // stays Active; its next visit confirms (or not) that it converged
            if (ord.on && lane == 0) atomicMin(knext + g, key);
            warp_push(ctl, &ctl->cnt[nslot], out, P.n_tiles, lane == 0, g, ord.on ? &ctl->kmin[nslot] : nullptr, key);
        } else {
            if (lane == 0) __stcg(P.tstate + g, (int)kSource);                    // Active -> Source
            const int prev = nbf >= 0 ? atomicCAS(P.tstate + nbf, (int)kDistant, (int)kActive) : (int)kSource;
            const bool act = prev == (int)kDistant;
            unsigned kf = kKeyInf;
            if (ord.on) {
                // key of the neighbour across face `lane`: the smallest value on that face
                const float sc = P.inst_scale[__ldcg(P.tile_inst + g)];
                float fm = __int_as_float(0x7f800000);
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    const unsigned k = __reduce_min_sync(kFull, key_enc(face_min<T, BX, BY, BZ>(~0u, v, f)));
                    if (lane == f) fm = key_dec(k);
                }
                kf = key_enc(fm * sc);
                if (act || prev == (int)kActive) atomicMin(knext + nbf, kf);
            }
            warp_push(ctl, &ctl->cnt[nslot], out, P.n_tiles, act, nbf, ord.on ? &ctl->kmin[nslot] : nullptr, kf);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- Step 3
// Recompute every tile once; a tile holding a non-source node whose root is
// below its value seeds the Remedy list (stamp 1, key = smallest such root).
// Nothing is written to phi.  Also clears both key parities.
template <class T, int BX, int BY, int BZ>
__device__ void detect_pass(const FwdParams<T> &P, T *sm, long long &st_flagged) {
    using G = TileGeom<BX, BY, BZ>;
    Ctl *ctl = P.ctl;
    const int lane = lane_id();
    for (int g = warp_global(); g < P.n_tiles; g += warps_total()) {
        const int nbf = lane < 6 ? __ldcg(P.tile_nb + 6 * g + lane) : -1;
        T v[G::NPL], tau[G::NPL];
        stage_tile<T, BX, BY, BZ>(P, sm, g, nbf, v, tau);
        bool low = false;
        float kmin = __int_as_float(0x7f800000);
#pragma unroll
        for (int m = 0; m < G::NPL; ++m) {
            if (!(tau[m] < T(0))) {
                const int c = G::sidx_of(lane + 32 * m);
                const T ax = vmin(sm[c - 1], sm[c + 1]);
                const T ay = vmin(sm[c - G::SX], sm[c + G::SX]);
                const T az = vmin(sm[c - G::SX * G::SY], sm[c + G::SX * G::SY]);
                const T u = local_solve<T>(ax, ay, az, tau[m]);
                if (u < v[m]) { low = true; kmin = fminf(kmin, (float)u); }
            }
        }
        const bool any = __any_sync(kFull, low);
        if (P.ordered) {
            const unsigned k = warp_min_key(kmin * P.inst_scale[__ldcg(P.tile_inst + g)]);
            if (lane == 0) {
                __stcg(P.tkey + g, any ? k : kKeyInf);
                __stcg(P.tkey + P.n_tiles + g, kKeyInf);
                if (any) atomicMin(&ctl->rkmin[0], k);
            }
        }
        if (any && lane == 0) {
            st_flagged++;
            atomicExch(P.tstamp + g, 1);
        }
        warp_push(ctl, &ctl->rcnt[0], P.list0, P.n_tiles, any && lane == 0, g);
        __syncwarp();
    }
}

// One pass over the Remedy list of loop iteration r (slot r % 3, stamp r+1).
template <class T, int BX, int BY, int BZ>
__device__ void remedy_pass(const FwdParams<T> &P, T *sm, int r, int n, unsigned kmin_cur, long long &st_tiles,
                            long long &st_sweeps, long long &st_def) {
    using G = TileGeom<BX, BY, BZ>;
    Ctl *ctl = P.ctl;
    const int nslot = (r + 1) % 3;
    const int *in = (r & 1) ? P.list1 : P.list0;
    int *out = (r & 1) ? P.list0 : P.list1;
    unsigned *kcur = P.tkey + (size_t)(r & 1) * P.n_tiles;
    unsigned *knext = P.tkey + (size_t)((r + 1) & 1) * P.n_tiles;
    const int lane = lane_id();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->rcnt[(r + 2) % 3] = 0;
        ctl->rkmin[(r + 2) % 3] = kKeyInf;
    }
    const OrderCtx ord = order_begin(P.ordered, kmin_cur);
    n = min(n, P.n_tiles);
    const int next_stamp = r + 2;
    for (int idx = warp_global(); idx < n; idx += warps_total()) {
        const int g = __ldcg(in + idx);
        unsigned key = kKeyInf;
        if (ord.on) {
            if (lane == 0) key = atomicExch(kcur + g, kKeyInf);
            key = __shfl_sync(kFull, key, 0);
            if (!order_visit(ord, key)) {        // deferred: listed again, not visited
                bool want = false;
                if (lane == 0) {
                    atomicMin(knext + g, key);
                    want = atomicExch(P.tstamp + g, next_stamp) != next_stamp;
                    st_def++;
                }
                warp_push(ctl, &ctl->rcnt[nslot], out, P.n_tiles, want, g, &ctl->rkmin[nslot], key);
                continue;
            }
        }
        const int nbf = lane < 6 ? __ldcg(P.tile_nb + 6 * g + lane) : -1;
        T v[G::NPL], tau[G::NPL];
        stage_tile<T, BX, BY, BZ>(P, sm, g, nbf, v, tau);
        unsigned mine;
        bool changed;
        const int s = relax_tile<T, BX, BY, BZ>(sm, v, tau, P.max_sweeps, mine, changed);
        write_back<T, BX, BY, BZ>(P, g, mine, v);
        const int fm = changed_faces<BX, BY, BZ>(mine);
        if (lane == 0) { st_tiles++; st_sweeps += s; }
        // The tile is relaxed to its local fixed point; a neighbour whose facing
        // boundary drops re-lists it.  Lanes 0-5 list the neighbour across face
        // `lane` when a node on that face dropped; lane 6 re-lists the tile
        // itself when the sweep cap stopped the relaxation early.
        int cand = -1;
        if (lane < 6 && (fm >> lane & 1)) cand = nbf;
        if (lane == 6 && changed && s >= P.max_sweeps) cand = g;
        unsigned kc = kKeyInf;
        if (ord.on) {
            const float sc = P.inst_scale[__ldcg(P.tile_inst + g)];
            float dm = __int_as_float(0x7f800000);
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                if (!(fm >> f & 1)) continue;                     // warp-uniform
                const unsigned k = __reduce_min_sync(kFull, key_enc(face_min<T, BX, BY, BZ>(mine, v, f)));
                if (lane == f) dm = key_dec(k);
            }
            kc = lane == 6 ? key : key_enc(dm * sc);
            if (cand >= 0) atomicMin(knext + cand, kc);
        }
        const bool want = cand >= 0 && atomicExch(P.tstamp + cand, next_stamp) != next_stamp;
        // a tile already listed for r+1 by another warp took its key through knext;
        // the list minimum must still see this key
        if (ord.on && cand >= 0 && !want) atomicMin(&ctl->rkmin[nslot], kc);
        warp_push(ctl, &ctl->rcnt[nslot], out, P.n_tiles, want, cand, ord.on ? &ctl->rkmin[nslot] : nullptr, kc);
        __syncwarp();
    }
}

// ---------------------------------------------------------------- kernels
// Descriptor upload (by-value parameter, so that the call can be captured).
__global__ void k_write_desc(InstDesc *desc, double *inst_acc, DescChunk chunk) {
    const int i = threadIdx.x;
    if (i < chunk.count) {
        desc[chunk.first + i] = chunk.d[i];
        inst_acc[2 * (chunk.first + i)] = 0.0;
        inst_acc[2 * (chunk.first + i) + 1] = 0.0;
    }
}

// 1/delta per instance for the ordered schedule: delta = order * (mean tile
// edge) * h / mean(F over passable nodes).
template <int BX, int BY, int BZ>
__global__ void k_scale(const InstDesc *desc, const double *inst_acc, float *inst_scale, int B, float order) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double edge = BZ == 1 ? 0.5 * (BX + BY) : (BX + BY + BZ) / 3.0;
    const double cnt = inst_acc[2 * b + 1], sum = inst_acc[2 * b];
    const double meanF = cnt > 0 ? sum / cnt : 0.0;
    double sc = meanF > 0 ? meanF / ((double)order * edge * desc[b].h) : 1.0;
    if (!(sc > 0) || !(sc < 1e30)) sc = 1.0;
    inst_scale[b] = (float)sc;
}

// Step 1a: bricked tau = h/F and phi = +inf; per-tile state and neighbour
// ids; control block.  One CTA of V threads per tile.
template <class T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(BX *BY *BZ) k_init(FwdParams<T> P) {
    using G = TileGeom<BX, BY, BZ>;
    __shared__ int s_b;
    const int g = blockIdx.x;
    if (threadIdx.x == 0) s_b = find_inst_by_tile(P.desc, P.B, g);
    __syncthreads();
    const InstDesc &d = P.desc[s_b];
    const long long l = g - d.tile_base;
    const int tx = (int)(l % d.tx), ty = (int)((l / d.tx) % d.ty), tz = (int)(l / ((long long)d.tx * d.ty));
    const int tid = threadIdx.x;
    const int i = tx * BX + tid % BX, j = ty * BY + (tid / BX) % BY, k = tz * BZ + tid / (BX * BY);
    T tau = Num<T>::inf();
    double fsum = 0.0, fcnt = 0.0;
    if (i < d.nx && j < d.ny && k < d.nz) {
        const T f = P.F[d.in_off + ((long long)k * d.ny + j) * d.nx + i];
        if (f > T(0)) { tau = T(d.h) / f; fsum = (double)f; fcnt = 1.0; }
    }
    P.tau_t[(size_t)g * G::V + tid] = tau;
    P.phi_t[(size_t)g * G::V + tid] = Num<T>::inf();
    if (tid == 0) {
        P.tile_inst[g] = s_b;
        P.tstate[g] = kDistant;
        P.tstamp[g] = 0;
        P.tkey[g] = kKeyInf;
        P.tkey[P.n_tiles + g] = kKeyInf;
    }
    if (P.ordered) {   // per-instance mean speed for the bucket width
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fsum += __shfl_xor_sync(0xffffffffu, fsum, o);
            fcnt += __shfl_xor_sync(0xffffffffu, fcnt, o);
        }
        if ((tid & 31) == 0 && fcnt > 0) {
            atomicAdd(P.inst_acc + 2 * s_b, fsum);
            atomicAdd(P.inst_acc + 2 * s_b + 1, fcnt);
        }
    }
    if (tid < 6) {
        int nb;
        switch (tid) {
            case 0: nb = tx > 0 ? g - 1 : -1; break;
            case 1: nb = tx + 1 < d.tx ? g + 1 : -1; break;
            case 2: nb = ty > 0 ? g - d.tx : -1; break;
            case 3: nb = ty + 1 < d.ty ? g + d.tx : -1; break;
            case 4: nb = tz > 0 ? g - d.tx * d.ty : -1; break;
            default: nb = tz + 1 < d.tz ? g + d.tx * d.ty : -1; break;
        }
        P.tile_nb[6 * g + tid] = nb;
    }
    if (g == 0 && tid < (int)(sizeof(Ctl) / sizeof(int))) {
        const int k0 = (int)(offsetof(Ctl, kmin) / sizeof(int)), k1 = (int)(offsetof(Ctl, rkmin) / sizeof(int)) + 3;
        reinterpret_cast<unsigned *>(P.ctl)[tid] = (tid >= k0 && tid < k1) ? kKeyInf : 0u;
    }
}

__device__ __forceinline__ void atomic_min_val(float *p, float v) {
    int old = __float_as_int(*(volatile float *)p);
    while (v < __int_as_float(old)) {
        const int prev = atomicCAS(reinterpret_cast<int *>(p), old, __float_as_int(v));
        if (prev == old) break;
        old = prev;
    }
}
__device__ __forceinline__ void atomic_min_val(double *p, double v) {
    unsigned long long old = __double_as_longlong(*(volatile double *)p);
    while (v < __longlong_as_double(old)) {
        const unsigned long long prev =
            atomicCAS(reinterpret_cast<unsigned long long *>(p), old, (unsigned long long)__double_as_longlong(v));
        if (prev == old) break;
        old = prev;
    }
}

// Step 1b: sources fixed (phi = value, tau = -1 marker); Active = the tiles
// that hold the sources' face neighbours (the source tile and, for a source on
// a tile face, the tile across that face).
template <class T, int BX, int BY, int BZ>
__global__ void k_sources(FwdParams<T> P) {
    using G = TileGeom<BX, BY, BZ>;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P.n_src) return;
    const int b = find_inst_by_src(P.desc, P.B, s);
    const InstDesc &d = P.desc[b];
    if (s < d.src_begin || s >= d.src_end) { atomicOr(&P.ctl->flags, kFlagBadSource); return; }
    const long long p = P.src_idx[s];
    const long long N = (long long)d.nx * d.ny * d.nz;
    if (p < 0 || p >= N) { atomicOr(&P.ctl->flags, kFlagBadSource); return; }
    const int i = (int)(p % d.nx), j = (int)((p / d.nx) % d.ny), k = (int)(p / ((long long)d.nx * d.ny));
    const int tx = i / BX, ty = j / BY, tz = k / BZ;
    const int g = (int)(d.tile_base + ((long long)tz * d.ty + ty) * d.tx + tx);
    const int loc = ((k % BZ) * BY + (j % BY)) * BX + (i % BX);
    atomic_min_val(P.phi_t + (size_t)g * G::V + loc, P.src_val[s]);
    P.tau_t[(size_t)g * G::V + loc] = T(-1);
    int cand[7];
    int nc = 0;
    cand[nc++] = g;
    if (i % BX == 0 && i > 0) cand[nc++] = g - 1;
    if (i % BX == BX - 1 && i + 1 < d.nx) cand[nc++] = g + 1;
    if (j % BY == 0 && j > 0) cand[nc++] = g - d.tx;
    if (j % BY == BY - 1 && j + 1 < d.ny) cand[nc++] = g + d.tx;
    if (k % BZ == 0 && k > 0) cand[nc++] = g - d.tx * d.ty;
    if (k % BZ == BZ - 1 && k + 1 < d.nz) cand[nc++] = g + d.tx * d.ty;
    const unsigned key = key_enc((float)P.src_val[s] * P.inst_scale[b]);
    for (int q = 0; q < nc; ++q) {
        if (P.ordered) {
            atomicMin(P.tkey + cand[q], key);
            atomicMin(&P.ctl->kmin[0], key);
        }
        if (atomicCAS(P.tstate + cand[q], (int)kDistant, (int)kActive) == (int)kDistant) {
            const int pos = atomicAdd(&P.ctl->cnt[0], 1);
            if (pos < P.n_tiles) P.list0[pos] = cand[q];
            else atomicOr(&P.ctl->flags, kFlagOverflow);
        }
    }
}

template <class T>
__device__ __forceinline__ void flush_stats(const FwdParams<T> &P, long long a, long long b, long long c,
                                            long long d, long long e) {
    if (lane_id() == 0) {
        if (e) atomicAdd((unsigned long long *)&P.ctl->tiles_deferred, (unsigned long long)e);
        if (a) atomicAdd((unsigned long long *)&P.ctl->tiles_update, (unsigned long long)a);
        if (b) atomicAdd((unsigned long long *)&P.ctl->tiles_flagged, (unsigned long long)b);
        if (c) atomicAdd((unsigned long long *)&P.ctl->tiles_remedy, (unsigned long long)c);
        if (d) atomicAdd((unsigned long long *)&P.ctl->sweeps, (unsigned long long)d);
    }
}

// resident CTAs per SM asked of the compiler (register budget per thread =
// 65536 / (32 * kWarpsPerCta * this)): more warps in flight for small tiles
template <class T, int BX, int BY, int BZ>
constexpr int min_ctas() {
    return sizeof(T) == 8 ? 2   // FP64 validation mode: registers over occupancy
           : TileGeom<BX, BY, BZ>::NPL <= 2 ? 6 : TileGeom<BX, BY, BZ>::NPL <= 4 ? 5
           : TileGeom<BX, BY, BZ>::NPL <= 8 ? 3 : 2;
}

template <class T, int BX, int BY, int BZ>
struct WarpSmem {
    T phi[kWarpsPerCta][TileGeom<BX, BY, BZ>::S];
};

// Steps 2 and 3 in one cooperative launch; iterations are separated by the
// bounded grid barrier.  Every warp reads the same list size after a
// barrier, so all CTAs leave the loops together.
template <class T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(32 * kWarpsPerCta, (min_ctas<T, BX, BY, BZ>())) k_persistent(FwdParams<T> P) {
    __shared__ WarpSmem<T, BX, BY, BZ> sm;
    __shared__ int s_n;
    __shared__ unsigned s_k;
    T *my = sm.phi[warp_in_cta()];
    init_stage<T, BX, BY, BZ>(my);
    Ctl *ctl = P.ctl;
    unsigned long long target = 0;
    long long t_upd = 0, t_flag = 0, t_rem = 0, sweeps = 0, deferred = 0;
    int it = 0, r = 0;
    for (;; ++it) {
        if (threadIdx.x == 0) { s_n = ld_volatile(&ctl->cnt[it % 3]); s_k = ld_volatile_u(&ctl->kmin[it % 3]); }
        __syncthreads();
        const int n = s_n;
        const unsigned kq = s_k;
        if (n == 0) break;
        if (it >= P.max_iters) { if (threadIdx.x == 0) atomicOr(&ctl->flags, kFlagCap); goto done; }
        update_pass<T, BX, BY, BZ>(P, my, it, n, kq, t_upd, sweeps, deferred);
        if (!grid_sync(ctl, target)) goto done;
    }
    if (P.skip_remedy) goto done;
    detect_pass<T, BX, BY, BZ>(P, my, t_flag);
    if (!grid_sync(ctl, target)) goto done;
    for (;; ++r) {
        if (threadIdx.x == 0) { s_n = ld_volatile(&ctl->rcnt[r % 3]); s_k = ld_volatile_u(&ctl->rkmin[r % 3]); }
        __syncthreads();
        const int n = s_n;
        const unsigned kq = s_k;
        if (n == 0) break;
        if (r >= P.max_iters) { if (threadIdx.x == 0) atomicOr(&ctl->flags, kFlagCap); goto done; }
        remedy_pass<T, BX, BY, BZ>(P, my, r, n, kq, t_rem, sweeps, deferred);
        if (!grid_sync(ctl, target)) goto done;
    }
done:
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->iters_update = it;
        ctl->iters_remedy = r;
    }
    flush_stats<T>(P, t_upd, t_flag, t_rem, sweeps, deferred);
}

// Host-loop schedule: one launch per iteration.
template <class T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(32 * kWarpsPerCta, (min_ctas<T, BX, BY, BZ>())) k_update_iter(FwdParams<T> P, int it) {
    __shared__ WarpSmem<T, BX, BY, BZ> sm;
    const int n = ld_volatile(&P.ctl->cnt[it % 3]);
    const unsigned kq = ld_volatile_u(&P.ctl->kmin[it % 3]);
    long long t = 0, s = 0, d = 0;
    init_stage<T, BX, BY, BZ>(sm.phi[warp_in_cta()]);
    update_pass<T, BX, BY, BZ>(P, sm.phi[warp_in_cta()], it, n, kq, t, s, d);
    flush_stats<T>(P, t, 0, 0, s, d);
}

template <class T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(32 * kWarpsPerCta, (min_ctas<T, BX, BY, BZ>())) k_detect(FwdParams<T> P) {
    __shared__ WarpSmem<T, BX, BY, BZ> sm;
    long long f = 0;
    init_stage<T, BX, BY, BZ>(sm.phi[warp_in_cta()]);
    detect_pass<T, BX, BY, BZ>(P, sm.phi[warp_in_cta()], f);
    flush_stats<T>(P, 0, f, 0, 0, 0);
}

template <class T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(32 * kWarpsPerCta, (min_ctas<T, BX, BY, BZ>())) k_remedy_iter(FwdParams<T> P, int r) {
    __shared__ WarpSmem<T, BX, BY, BZ> sm;
    const int n = ld_volatile(&P.ctl->rcnt[r % 3]);
    const unsigned kq = ld_volatile_u(&P.ctl->rkmin[r % 3]);
    long long t = 0, s = 0, d = 0;
    init_stage<T, BX, BY, BZ>(sm.phi[warp_in_cta()]);
    remedy_pass<T, BX, BY, BZ>(P, sm.phi[warp_in_cta()], r, n, kq, t, s, d);
    flush_stats<T>(P, 0, 0, t, s, d);
}

// Output: bricked phi -> caller's row-major phi.  One CTA of V threads per tile.
template <class T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(BX *BY *BZ) k_unpack(FwdParams<T> P) {
    using G = TileGeom<BX, BY, BZ>;
    const int g = blockIdx.x;
    const int b = P.tile_inst[g];
    const InstDesc &d = P.desc[b];
    const long long l = g - d.tile_base;
    const int tx = (int)(l % d.tx), ty = (int)((l / d.tx) % d.ty), tz = (int)(l / ((long long)d.tx * d.ty));
    const int tid = threadIdx.x;
    const int i = tx * BX + tid % BX, j = ty * BY + (tid / BX) % BY, k = tz * BZ + tid / (BX * BY);
    if (i < d.nx && j < d.ny && k < d.nz)
        P.phi_out[d.out_off + ((long long)k * d.ny + j) * d.nx + i] = P.phi_t[(size_t)g * G::V + tid];
}

}  // namespace eik
