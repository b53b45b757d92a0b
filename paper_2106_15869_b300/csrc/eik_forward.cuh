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

#include <type_traits>

#include "eik_common.cuh"

namespace eik {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerCta = 8;

// A tile kept by the classification of a two-phase iteration: {tile, key},
// and its record (neighbours, instance, key scale) as in tile_nb.
struct VisitRec {
    int4 head;
    int4 r0, r1;
};

template <class T>
struct FwdParams {
    const InstDesc *desc;
    int B;
    int n_tiles;                 // total tiles over all instances
    int *tile_inst;
    int *tile_nb;                // [n_tiles][8]: neighbour tile ids (-1 outside) across -x,+x,-y,+y,-z,+z,
                                 // the instance, and (ordered schedule) the instance's key scale
    int *tstate;
    int *tstamp;
    unsigned *tkey;              // [2][n_tiles] encoded list keys (ordered schedule)
    float *inst_scale;           // [B] 1/delta of each instance (ordered schedule)
    ScalePart *scale_part;       // [B][scale_chunks(B)] partial slowness statistics (k_scale)
    int *scale_done;             // [B] k_scale CTAs finished per instance
    float *tile_fstat;           // [n_tiles][2] sum of 1/F and count over passable nodes (delta)
    int ordered;                 // 1 = bucketed order of the Step-3 (and FIM) lists; keys are kept
    int ordered_update;          // 1 = bucketed order of the Step-2 lists too
    float order;                 // bucket width in tile-crossing times
    int *list0, *list1;
    VisitRec *vlist;             // the tiles kept by the classification of a two-phase iteration
    T *phi_t, *tau_t;
    Ctl *ctl;
    long long max_iters;
    Metric<T> mt;                // axis weights of unequal spacings
    int skip_remedy;
    int fim;                     // 1 = the fast iterative method of Sec. 2.3 (one neighbour-check loop)
    int one_visit;               // Step 2: a visit whose relaxation converged moves the tile to Source
    int max_sweeps;              // cap on in-tile sweeps per visit
    const T *F;                  // packed input speeds
    const long long *src_idx;
    const T *src_val;
    long long n_src;
    T *phi_out;                  // packed output
    unsigned long long wait_ns;  // bound on every device wait of the call
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
            if ((unsigned)n < (unsigned)P.n_tiles) hv = __ldcg(P.phi_t + (size_t)n * G::V + src);
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
                                          const Metric<T> &mt, unsigned &mine, bool &first_changed) {
    using G = TileGeom<BX, BY, BZ>;
    const int lane = lane_id();
    mine = 0;
    first_changed = false;
    // the sweeps, with the spacing case (equal or unequal) fixed for the whole loop
    auto sweep_loop = [&](auto aniso) {
        unsigned act = G::NPL >= 32 ? ~0u : ((1u << G::NPL) - 1u);
        int s = 0;
        for (;;) {
            unsigned ch = 0;
#pragma unroll
            for (int m = 0; m < G::NPL; ++m) {
                if (act >> m & 1) {
                    const int c = G::sidx_of(lane + 32 * m);
                    const T ax = vmin(sm[c - 1], sm[c + 1]);
                    const T ay = vmin(sm[c - G::SX], sm[c + G::SX]);
                    const T az = vmin(sm[c - G::SX * G::SY], sm[c + G::SX * G::SY]);
                    const T u = node_solve_fixed<decltype(aniso)::value>(ax, ay, az, tau[m], mt);
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
    };
    return mt.aniso ? sweep_loop(std::true_type{}) : sweep_loop(std::false_type{});
}

// Step-3 listing test.  A node p of a tile that dropped to value u can lower
// the node q across face f of the neighbour tile only if u < phi(q): otherwise
// the term ((phi - u)^+)^2 of q's eq. (6) stays 0 at phi(q), so q's root
// cannot fall below phi(q) (a neighbour tile at its fixed point stays there;
// one that is not is listed already by whatever moved it).  The staged halo
// holds phi(q) as it was when the visit began, never below its current value,
// so the test can only list more.  Of fb (the faces of the node at staged slot
// c), the faces across which value u lies below the halo.
template <class T, int BX, int BY, int BZ>
__device__ __forceinline__ int below_halo(const T *sm, int c, T u, int fb) {
    using G = TileGeom<BX, BY, BZ>;
    int r = 0;
    if ((fb & 1) && u < sm[c - 1]) r |= 1;
    if ((fb & 2) && u < sm[c + 1]) r |= 2;
    if ((fb & 4) && u < sm[c - G::SX]) r |= 4;
    if ((fb & 8) && u < sm[c + G::SX]) r |= 8;
    if ((fb & 16) && u < sm[c - G::SX * G::SY]) r |= 16;
    if ((fb & 32) && u < sm[c + G::SX * G::SY]) r |= 32;
    return r;
}

// Faces across which a dropped node of the warp's tile (bit m of `mine`:
// node lane + 32 m) lies below the staged halo (below_halo), warp-reduced.
template <class T, int BX, int BY, int BZ>
__device__ __forceinline__ int lowering_faces(unsigned mine, const T (&v)[TileGeom<BX, BY, BZ>::NPL], const T *sm) {
    using G = TileGeom<BX, BY, BZ>;
    int f = 0;
#pragma unroll
    for (int m = 0; m < G::NPL; ++m)
        if (mine >> m & 1) {
            const int q = lane_id() + 32 * m;
            f |= below_halo<T, BX, BY, BZ>(sm, G::sidx_of(q), v[m], G::faces_of(q));
        }
    return (int)__reduce_or_sync(kFull, (unsigned)f);
}

template <class T, int BX, int BY, int BZ>
__device__ __forceinline__ void write_back(const FwdParams<T> &P, int g, unsigned mine,
                                           const T (&v)[TileGeom<BX, BY, BZ>::NPL]) {
    using G = TileGeom<BX, BY, BZ>;
    T *pg = P.phi_t + (size_t)g * G::V;
#pragma unroll
    for (int m = 0; m < G::NPL; ++m)
        if (mine >> m & 1) {
            dbg_nan(P.ctl, v[m]);
            __stcg(pg + lane_id() + 32 * m, v[m]);
        }
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
// others to the next list unvisited.  The bucket width starts at one unit and adapts
// (adapt_window) when most of a list is deferred.  The sets and their rules
// are those of Algorithm 2; only the iteration in which a listed tile is
// visited changes,
// and the fixed point reached does not depend on that (the discrete solution
// is unique).  Keys live in two parities: pushes for iteration it+1 write
// tkey[(it+1)&1], the visit in iteration it reads and clears tkey[it&1].
struct OrderCtx {
    bool on;
    unsigned kmin;      // smallest key listed for this iteration (encoded)
    float theta;        // visit iff key < theta (or every key is +inf)
};

__device__ __forceinline__ OrderCtx order_begin(bool on, unsigned kmin, float width) {
    OrderCtx o;
    o.on = on;
    o.kmin = on ? kmin : kKeyInf;
    o.theta = key_dec(o.kmin) + width;
    return o;
}

__device__ __forceinline__ bool order_visit(const OrderCtx &o, unsigned key) {
    return !o.on || o.kmin == kKeyInf || key_dec(key) < o.theta;
}

// warp min of one float per lane, encoded
__device__ __forceinline__ unsigned warp_min_key(float k) { return __reduce_min_sync(kFull, key_enc(k)); }

// per-face minimum over this lane's nodes selected by `sel`, for face f; with
// a staged block `sm`, only over the nodes below the halo across f (below_halo)
template <class T, int BX, int BY, int BZ>
__device__ __forceinline__ float face_min(unsigned sel, const T (&v)[TileGeom<BX, BY, BZ>::NPL], int f,
                                          const T *sm = nullptr) {
    using G = TileGeom<BX, BY, BZ>;
    float m = __int_as_float(0x7f800000);
#pragma unroll
    for (int q = 0; q < G::NPL; ++q) {
        const int n = lane_id() + 32 * q;
        if (!(sel >> q & 1) || !(G::faces_of(n) >> f & 1)) continue;
        if (sm && !below_halo<T, BX, BY, BZ>(sm, G::sidx_of(n), v[q], 1 << f)) continue;
        m = fminf(m, (float)v[q]);
    }
    return m;
}

// ---------------------------------------------------------------- Step 2
// One pass over the Active list of iteration `it` (slot it % 3).
template <class T, int BX, int BY, int BZ>
__device__ void update_pass(const FwdParams<T> &P, T *sm, int it, int n, unsigned kmin_cur, float width,
                            int *s_visits, long long &st_tiles,
                            long long &st_sweeps, long long &st_def) {
    using G = TileGeom<BX, BY, BZ>;
    Ctl *ctl = P.ctl;
    const int nslot = (it + 1) % 3;
    const int *in = (it & 1) ? P.list1 : P.list0;
    int *out = (it & 1) ? P.list0 : P.list1;
    unsigned *kcur = P.tkey + (size_t)(it & 1) * P.n_tiles;
    unsigned *knext = P.tkey + (size_t)((it + 1) & 1) * P.n_tiles;
    const int lane = lane_id();
    const OrderCtx ord = order_begin(P.ordered_update, kmin_cur, width);
    n = min(n, P.n_tiles);                       // n > n_tiles only after an overflow
    for (int idx = warp_global(); idx < n; idx += warps_total()) {
        const int g = __ldcg(in + idx);
        if (dbg_bad_tile(ctl, g, P.n_tiles)) continue;             // warp-uniform
        // one round trip: the tile record (lanes 0-7) and its key (lane 8)
        const int rec = lane < 8 ? __ldcg(P.tile_nb + 8 * g + lane) : (lane == 8 && ord.on ? (int)__ldcg(kcur + g) : -1);
        const int nbf = lane < 6 ? rec : -1;
        const float sc = __int_as_float(__shfl_sync(kFull, rec, 7));
        unsigned key = (unsigned)__shfl_sync(kFull, rec, 8);
        if (ord.on) {
            if (lane == 8) __stcg(kcur + g, kKeyInf);   // no one writes this parity in this iteration
            if (!order_visit(ord, key)) {        // deferred: listed again, not visited
                if (lane == 0) {
                    atomicMin(knext + g, key);
                    st_def++;
                }
                warp_push(ctl, &ctl->cnt[nslot], out, P.n_tiles, lane == 0, g, &ctl->kmin[nslot], key);
                continue;
            }
        }
        T v[G::NPL], tau[G::NPL];
        stage_tile<T, BX, BY, BZ>(P, sm, g, nbf, v, tau);
        unsigned mine;
        bool changed;
        const int s = relax_tile<T, BX, BY, BZ>(sm, v, tau, P.max_sweeps, P.mt, mine, changed);
        write_back<T, BX, BY, BZ>(P, g, mine, v);
        if (lane == 0) { st_tiles++; st_sweeps += s; atomicAdd(s_visits, 1); }
        if (changed && (!P.one_visit || s >= P.max_sweeps)) {
            // stays Active; its next visit confirms (or not) that it converged
            if (ord.on && lane == 0) atomicMin(knext + g, key);
            warp_push(ctl, &ctl->cnt[nslot], out, P.n_tiles, lane == 0, g, ord.on ? &ctl->kmin[nslot] : nullptr, key);
        } else {
            if (lane == 0) __stcg(P.tstate + g, (int)kSource);                    // Active -> Source
            const int prev = (unsigned)nbf < (unsigned)P.n_tiles ? atomicCAS(P.tstate + nbf, (int)kDistant, (int)kActive)
                                                                 : (int)kSource;
            const bool act = prev == (int)kDistant;
            unsigned kf = kKeyInf;
            if (ord.on) {
                // key of the neighbour across face `lane`: the smallest value on that face
                float fm = __int_as_float(0x7f800000);
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    const unsigned k = __reduce_min_sync(kFull, key_enc(face_min<T, BX, BY, BZ>(~0u, v, f)));
                    if (lane == f) fm = key_dec(k);
                }
                kf = scaled_key(fm, sc);
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
        const int rec = lane < 8 ? __ldcg(P.tile_nb + 8 * g + lane) : -1;
        const int nbf = lane < 6 ? rec : -1;
        const float sc = __int_as_float(__shfl_sync(kFull, rec, 7));
        T v[G::NPL], tau[G::NPL];
        stage_tile<T, BX, BY, BZ>(P, sm, g, nbf, v, tau);
        bool low = false;
        float kmin = __int_as_float(0x7f800000);
        auto check = [&](auto aniso) {
#pragma unroll
            for (int m = 0; m < G::NPL; ++m) {
                const int c = G::sidx_of(lane + 32 * m);
                const T ax = vmin(sm[c - 1], sm[c + 1]);
                const T ay = vmin(sm[c - G::SX], sm[c + G::SX]);
                const T az = vmin(sm[c - G::SX * G::SY], sm[c + G::SX * G::SY]);
                const T u = node_solve_fixed<decltype(aniso)::value>(ax, ay, az, tau[m], P.mt);
                if (u < v[m]) { low = true; kmin = fminf(kmin, (float)u); }
            }
        };
        if (P.mt.aniso) check(std::true_type{}); else check(std::false_type{});
        const bool any = __any_sync(kFull, low);
        if (P.ordered) {
            const unsigned k = __reduce_min_sync(kFull, scaled_key(kmin, sc));
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
__device__ void remedy_pass(const FwdParams<T> &P, T *sm, int r, int n, unsigned kmin_cur, float width,
                            int *s_visits, long long &st_tiles,
                            long long &st_sweeps, long long &st_def) {
    using G = TileGeom<BX, BY, BZ>;
    Ctl *ctl = P.ctl;
    const int nslot = (r + 1) % 3;
    const int *in = (r & 1) ? P.list1 : P.list0;
    int *out = (r & 1) ? P.list0 : P.list1;
    unsigned *kcur = P.tkey + (size_t)(r & 1) * P.n_tiles;
    unsigned *knext = P.tkey + (size_t)((r + 1) & 1) * P.n_tiles;
    const int lane = lane_id();
    const OrderCtx ord = order_begin(P.ordered, kmin_cur, width);
    n = min(n, P.n_tiles);
    const int next_stamp = r + 2;
    for (int idx = warp_global(); idx < n; idx += warps_total()) {
        const int g = __ldcg(in + idx);
        if (dbg_bad_tile(ctl, g, P.n_tiles)) continue;             // warp-uniform
        const int rec = lane < 8 ? __ldcg(P.tile_nb + 8 * g + lane) : (lane == 8 && ord.on ? (int)__ldcg(kcur + g) : -1);
        const int nbf = lane < 6 ? rec : -1;
        const float sc = __int_as_float(__shfl_sync(kFull, rec, 7));
        unsigned key = (unsigned)__shfl_sync(kFull, rec, 8);
        if (ord.on) {
            if (lane == 8) __stcg(kcur + g, kKeyInf);
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
        T v[G::NPL], tau[G::NPL];
        stage_tile<T, BX, BY, BZ>(P, sm, g, nbf, v, tau);
        unsigned mine;
        bool changed;
        const int s = relax_tile<T, BX, BY, BZ>(sm, v, tau, P.max_sweeps, P.mt, mine, changed);
        write_back<T, BX, BY, BZ>(P, g, mine, v);
        const int fm = lowering_faces<T, BX, BY, BZ>(mine, v, sm);
        if (lane == 0) { st_tiles++; st_sweeps += s; atomicAdd(s_visits, 1); }
        // The tile is relaxed to its local fixed point; a neighbour whose facing
        // boundary drops re-lists it.  Lanes 0-5 list the neighbour across face
        // `lane` when a node on that face dropped below the node across it;
        // lane 6 re-lists the tile itself when the sweep cap stopped the
        // relaxation early.
        int cand = -1;
        if (lane < 6 && (fm >> lane & 1) && (unsigned)nbf < (unsigned)P.n_tiles) cand = nbf;
        if (lane == 6 && changed && s >= P.max_sweeps) cand = g;
        unsigned kc = kKeyInf;
        if (ord.on) {
            float dm = __int_as_float(0x7f800000);
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                if (!(fm >> f & 1)) continue;                     // warp-uniform
                const unsigned k = __reduce_min_sync(kFull, key_enc(face_min<T, BX, BY, BZ>(mine, v, f, sm)));
                if (lane == f) dm = key_dec(k);
            }
            kc = lane == 6 ? key : scaled_key(dm, sc);
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

}  // namespace eik
