// eik_group.cuh -- latency mode of the tile passes: a group of threads per tile.
//
// In an iteration with a short list (the usual case in Step 2, where the
// Active set is a thin band) the iteration time is the latency of one tile
// visit, not throughput.  There, a group of GT threads (GT = min(V, 256))
// owns a tile with V/GT nodes per thread (1 or 2), so a sweep costs one or
// two local solves plus a named barrier instead of V/32 solves in a row;
// the group's OR-barrier is the convergence flag.  The rules applied are
// exactly those of the warp passes in eik_forward.cuh; an iteration uses one
// mode or the other for all its tiles (every CTA sees the same list size).
#pragma once

#include <type_traits>

#include "eik_forward.cuh"

namespace eik {

// threads per latency-mode group (at most a CTA).  Measured on B300: 256
// threads (one node per thread for 16x16x1 tiles, two for 8x8x8) against 128
// is 1.3-1.5x faster on 2D grids and equal on 3D; 64 is slower on both.
constexpr int kGroupThreads = 256;
static_assert(kGroupThreads <= 32 * kWarpsPerCta, "a group fits in a CTA");
// groups of the latency-only persistent kernel in iterations with more visits
// expected than 256-thread groups: twice as many groups of half the size
constexpr int kSmallGroupThreads = 128;
// and in iterations with many more visits than that: groups of 64 threads, a
// whole z column of an 8x8x8 tile per thread (a sweep is Gauss-Seidel along
// the column), four times as many groups as 256-thread ones in flight
constexpr int kColumnGroupThreads = 64;
constexpr int kColumnGroupFactor = 4;     // expected visits above this many 256-thread groups

template <int BX, int BY, int BZ, int MaxGT = kGroupThreads>
struct GroupGeom {
    using G = TileGeom<BX, BY, BZ>;
    static constexpr int CTA = 32 * kWarpsPerCta;
    static constexpr int GT = G::V >= MaxGT ? MaxGT : G::V;   // threads per group
    static constexpr int NG = CTA / GT;                    // groups per CTA
    static constexpr int NPT = G::V / GT;                  // nodes per thread
    static_assert(NG <= kWarpsPerCta && NG <= 8, "one staged block per group");
    // Node of slot m of group thread gt.  Where the tile's (x, y) columns
    // divide the group, a thread owns NPT consecutive z planes of one column,
    // and a sweep relaxes them in ascending z: within the thread a sweep is
    // Gauss-Seidel along z, so a front moving up the tile crosses NPT planes
    // per sweep instead of one (measured: 10 % fewer sweeps on the 3D
    // workloads, 5 % less time; group_visit picks descending z for fronts
    // coming from above).  Otherwise slot m is node gt + GT m.
    static constexpr int PLANE = BX * BY;
    static constexpr bool ZSEG = GT % PLANE == 0 && (GT / PLANE) * NPT == BZ;
    static __device__ __forceinline__ int node(int gt, int m) {
        if constexpr (ZSEG) return gt % PLANE + PLANE * ((gt / PLANE) * NPT + m);
        else return gt + GT * m;
    }
};

// Staged positions of a tile's halo elements for the group passes, one packed
// word per element (slot in the padded block, node of the neighbour tile,
// face): a visit reads one word per element instead of redoing the index
// arithmetic of TileGeom::halo_of.  Filled once per launch (halo_table_fill,
// then a CTA barrier) by every kernel that runs group passes.
template <int BX, int BY, int BZ>
__device__ __forceinline__ unsigned *halo_table() {
    __shared__ unsigned t[TileGeom<BX, BY, BZ>::HALO_LOADED];
    return t;
}
template <int BX, int BY, int BZ>
__device__ __forceinline__ void halo_table_fill() {
    using G = TileGeom<BX, BY, BZ>;
    static_assert(G::S <= 2048 && G::V <= 1024, "slot and node fit their fields");
    unsigned *t = halo_table<BX, BY, BZ>();
    for (int h = threadIdx.x; h < G::HALO_LOADED; h += blockDim.x) {
        int f, slot, src;
        G::halo_of(h, f, slot, src);
        t[h] = (unsigned)slot | (unsigned)src << 11 | (unsigned)f << 21;
    }
}

struct GroupCtl {
    int tile;
    unsigned key;
    int nb[6];
    float scale;
    int fmask;
    unsigned fmin[6];
};

__device__ __forceinline__ void group_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ int group_sync_or(int id, int n, int pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 q, %1, 0;\n\tbar.red.or.pred p, %2, %3, q;\n\tselp.s32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"(pred), "r"(id), "r"(n)
        : "memory");
    return r;
}

// Stage a tile for the group and relax it; returns the sweep count.
template <class T, int BX, int BY, int BZ, int GTM = kGroupThreads>
__device__ __forceinline__ int group_visit(const FwdParams<T> &P, T *sm, const GroupCtl &gc, int g, int gt, int bid,
                                           T (&v)[GroupGeom<BX, BY, BZ, GTM>::NPT], unsigned &mine,
                                           bool &first_changed) {
    using G = TileGeom<BX, BY, BZ>;
    using GG = GroupGeom<BX, BY, BZ, GTM>;
    T tau[GG::NPT];
    int c[GG::NPT];
    const T *pg = P.phi_t + (size_t)g * G::V;
    const T *tg = P.tau_t + (size_t)g * G::V;
#pragma unroll
    for (int m = 0; m < GG::NPT; ++m) {
        const int q = GG::node(gt, m);
        v[m] = __ldcg(pg + q);
        tau[m] = __ldcg(tg + q);
        c[m] = G::sidx_of(q);
        sm[c[m]] = v[m];
    }
    const unsigned *ht = halo_table<BX, BY, BZ>();
    for (int h = gt; h < G::HALO_LOADED; h += GG::GT) {
        const unsigned e = ht[h];
        const int slot = (int)(e & 2047u), src = (int)(e >> 11 & 1023u), n = gc.nb[e >> 21];
        sm[slot] = (unsigned)n < (unsigned)P.n_tiles ? __ldcg(P.phi_t + (size_t)n * G::V + src) : Num<T>::inf();
    }
    group_sync(bid, GG::GT);
    // z order of the segments: descending when the front comes from above
    // (the halo above the thread's column is lower than the one below, by a
    // majority of the warp, so that the warp does not diverge)
    bool down = false;
    if constexpr (GG::ZSEG && GG::NPT > 1) {
        const int col = G::sidx_of(gt % GG::PLANE);          // the column's node z = 0
        const T below = sm[col - G::SX * G::SY], above = sm[col + BZ * G::SX * G::SY];
        down = __popc(__ballot_sync(kFull, above < below)) > 16;
    }
    mine = 0;
    first_changed = false;
    // the sweeps, with the spacing case (equal or unequal) fixed for the whole loop
    auto sweep_loop = [&](auto aniso) {
        int s = 0;
        for (;;) {
            unsigned ch = 0;
            auto relax = [&](int m) {
                const T ax = vmin(sm[c[m] - 1], sm[c[m] + 1]);
                const T ay = vmin(sm[c[m] - G::SX], sm[c[m] + G::SX]);
                // z neighbours inside the thread's own segment come from registers (no
                // shared-memory round trip on the Gauss-Seidel chain; 1-2 % faster)
                T zlo, zhi;
                if constexpr (GG::ZSEG) {
                    zlo = m > 0 ? v[m > 0 ? m - 1 : 0] : sm[c[m] - G::SX * G::SY];
                    zhi = m + 1 < GG::NPT ? v[m + 1 < GG::NPT ? m + 1 : m] : sm[c[m] + G::SX * G::SY];
                } else {
                    zlo = sm[c[m] - G::SX * G::SY];
                    zhi = sm[c[m] + G::SX * G::SY];
                }
                const T az = vmin(zlo, zhi);
                const T u = node_solve_fixed<decltype(aniso)::value>(ax, ay, az, tau[m], P.mt);
                if (u < v[m]) { v[m] = u; sm[c[m]] = u; ch |= 1u << m; }
            };
            if (down) {
#pragma unroll
                for (int m = GG::NPT - 1; m >= 0; --m) relax(m);
            } else {
#pragma unroll
                for (int m = 0; m < GG::NPT; ++m) relax(m);
            }
            mine |= ch;
            ++s;
            const int any = group_sync_or(bid, GG::GT, ch != 0);
            if (s == 1) first_changed = any != 0;
            if (!any || s >= P.max_sweeps) break;
        }
        return s;
    };
    const int s = P.mt.aniso ? sweep_loop(std::true_type{}) : sweep_loop(std::false_type{});
#pragma unroll
    for (int m = 0; m < GG::NPT; ++m)
        if (mine >> m & 1) {
            dbg_nan(P.ctl, v[m]);
            __stcg(P.phi_t + (size_t)g * G::V + GG::node(gt, m), v[m]);
        }
    return s;
}

// Thread 0 of the group: the record (neighbours, key scale) of tile g.
__device__ __forceinline__ void group_set(GroupCtl &gc, int g, unsigned key, int4 r0, int4 r1) {
    gc.tile = g;
    gc.key = key;
    gc.nb[0] = r0.x; gc.nb[1] = r0.y; gc.nb[2] = r0.z; gc.nb[3] = r0.w; gc.nb[4] = r1.x; gc.nb[5] = r1.y;
    gc.scale = __int_as_float(r1.w);
    gc.fmask = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) gc.fmin[f] = kKeyInf;
}
template <class T>
__device__ __forceinline__ void group_fetch(const FwdParams<T> &P, GroupCtl &gc, int g, unsigned key) {
    group_set(gc, g, key, __ldcg(reinterpret_cast<const int4 *>(P.tile_nb + 8 * g)),
              __ldcg(reinterpret_cast<const int4 *>(P.tile_nb + 8 * g + 4)));
}

// per-node face bits of node q
template <int BX, int BY, int BZ>
__device__ __forceinline__ int node_faces_q(int q) { return TileGeom<BX, BY, BZ>::faces_of(q); }

// Face statistics of a visited tile over the nodes of the group selected by
// `sel` (bit m: the thread's node m): the faces holding a selected node
// (gc.fmask) and, per face, the smallest selected value as a key (gc.fmin).
// With the staged block `sm` (Step 3), a node counts for a face only if it
// lies below the halo value across it (below_halo).  Each thread reduces its
// own nodes, each warp reduces its lanes, and one lane per warp updates the
// shared record: a handful of shared atomics per visit instead of one per
// face node, which serialised on six addresses.  Every lane of the group's
// warps calls it.
template <class T, int BX, int BY, int BZ, int GTM>
__device__ __forceinline__ void group_face_stats(GroupCtl &gc, int gt, const T (&v)[GroupGeom<BX, BY, BZ, GTM>::NPT],
                                                 unsigned sel, bool want_mask, bool want_min,
                                                 const T *sm = nullptr) {
    using GG = GroupGeom<BX, BY, BZ, GTM>;
    float lm[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) lm[f] = Num<float>::inf();
    unsigned bits = 0;
#pragma unroll
    for (int m = 0; m < GG::NPT; ++m) {
        if (!(sel >> m & 1)) continue;
        const int q = GG::node(gt, m);
        int fb = node_faces_q<BX, BY, BZ>(q);
        if (sm) fb = below_halo<T, BX, BY, BZ>(sm, TileGeom<BX, BY, BZ>::sidx_of(q), v[m], fb);
        bits |= (unsigned)fb;
#pragma unroll
        for (int f = 0; f < 6; ++f)
            if (fb >> f & 1) lm[f] = fminf(lm[f], (float)v[m]);
    }
    const bool lead = lane_id() == 0;
    if (want_mask) {
        const unsigned b = __reduce_or_sync(kFull, bits);
        if (lead && b) atomicOr(&gc.fmask, (int)b);
    }
    if (want_min) {
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const unsigned k = __reduce_min_sync(kFull, key_enc(lm[f]));
            if (lead && k != kKeyInf) atomicMin(&gc.fmin[f], k);
        }
    }
}

// Per-group queue of the tiles a group visits from the chunk of the list it took.
constexpr int kQueueRec = 4;                           // queued tiles whose records the classification loads
struct GroupQueue {
    int tile[kGroupThreads];
    unsigned key[kGroupThreads];
    int4 rec[kQueueRec][2];
    int n;
    int base;
};

// Start of a group's next chunk of the list.  The first chunk of every group
// is static (its index among the launch's groups), the others come from a
// shared counter that starts after all the first chunks: the first grab of an
// iteration costs no atomic round trip, and a group whose first chunk lies
// past the end of the list learns so without one.
__device__ __forceinline__ int grab_chunk(int *grab, bool first, int group, int groups, int chunk) {
    return first ? group * chunk : groups * chunk + atomicAdd(grab, chunk);
}

// List entries per grab: about one visit per chunk at the previous
// iteration's visit rate (deferred entries are cheap, visits are not), at most
// n / (2 groups) so that every group gets work, at most one per thread.
__device__ __forceinline__ int group_chunk(int n, int visited_prev, int listed_prev, int groups, int gt) {
    int c = (listed_prev > 0 && visited_prev > 0) ? listed_prev / visited_prev : n;
    c = min(c, n / (2 * groups));
    return max(1, min(c, gt));
}

// Visit the tile the group fetched into gc and update the lists: Step 2 (the
// tile stays Active after a visit that changed it, else joins Source and
// activates its Distant face neighbours) or Step 3 (`remedy`: the face
// neighbours whose halo dropped are listed, the tile itself if the sweep cap
// stopped it).
template <class T, int BX, int BY, int BZ, bool remedy, int GTM>
__device__ __forceinline__ void visit_and_list(const FwdParams<T> &P, T *sm, GroupCtl &gc, int gt, int bid,
                                               const OrderCtx &ord, unsigned *knext, int *out, int *cnt_next,
                                               unsigned *kmin_next, int next_stamp, int *s_visits,
                                               long long &st_tiles, long long &st_sweeps) {
    using GG = GroupGeom<BX, BY, BZ, GTM>;
    Ctl *ctl = P.ctl;
    const int g = gc.tile;
    const unsigned key = gc.key;
    T v[GG::NPT];
    unsigned mine;
    bool changed;
    const int s = group_visit<T, BX, BY, BZ, GTM>(P, sm, gc, g, gt, bid, v, mine, changed);
    if (gt == 0) { st_tiles++; st_sweeps += s; atomicAdd(s_visits, 1); }
    if (!remedy) {
        if (changed && (!P.one_visit || s >= P.max_sweeps)) {
            // stays Active; its next visit confirms (or not) that it converged
            if (gt < 32) {
                if (ord.on && gt == 0) atomicMin(knext + g, key);
                warp_push(ctl, cnt_next, out, P.n_tiles, gt == 0, g, ord.on ? kmin_next : nullptr, key);
            }
        } else {
            // converged: Active -> Source, Distant face neighbours become Active
            if (ord.on) {
                group_face_stats<T, BX, BY, BZ, GTM>(gc, gt, v, ~0u, false, true);
                group_sync(bid, GG::GT);
            }
            if (gt < 32) {
                if (gt == 0) __stcg(P.tstate + g, (int)kSource);
                const int nbf = gt < 6 && (unsigned)gc.nb[gt] < (unsigned)P.n_tiles ? gc.nb[gt] : -1;
                const int prev = nbf >= 0 ? atomicCAS(P.tstate + nbf, (int)kDistant, (int)kActive) : (int)kSource;
                const bool act = prev == (int)kDistant;
                unsigned kf = kKeyInf;
                if (ord.on && nbf >= 0) {
                    kf = scaled_key(key_dec(gc.fmin[gt]), gc.scale);
                    if (act || prev == (int)kActive) atomicMin(knext + nbf, kf);
                }
                warp_push(ctl, cnt_next, out, P.n_tiles, act, nbf, ord.on ? kmin_next : nullptr, kf);
            }
        }
    } else {
        // faces where a node dropped below the node across, and (ordered) the smallest such value on each
        group_face_stats<T, BX, BY, BZ, GTM>(gc, gt, v, mine, true, ord.on, sm);
        group_sync(bid, GG::GT);
        if (gt < 32) {
            const int fm = gc.fmask;
            int cand = -1;
            if (gt < 6 && (fm >> gt & 1) && (unsigned)gc.nb[gt] < (unsigned)P.n_tiles) cand = gc.nb[gt];
            if (gt == 6 && changed && s >= P.max_sweeps) cand = g;
            unsigned kc = kKeyInf;
            if (ord.on && cand >= 0) {
                kc = gt == 6 ? key : scaled_key(key_dec(gc.fmin[gt]), gc.scale);
                atomicMin(knext + cand, kc);
            }
            const bool want = cand >= 0 && atomicExch(P.tstamp + cand, next_stamp) != next_stamp;
            if (ord.on && cand >= 0 && !want) atomicMin(kmin_next, kc);
            warp_push(ctl, cnt_next, out, P.n_tiles, want, cand, ord.on ? kmin_next : nullptr, kc);
        }
    }
    group_sync(bid, GG::GT);                           // the visit is done with gc
}

// Latency-mode iteration over a list: every thread group takes chunks of the
// list from a shared counter (dynamic balance: visits differ in length by an
// order of magnitude), classifies a chunk with all its threads at once (a
// deferred entry is listed again on the spot), queues the tiles to visit and
// visits them one by one.  `remedy` selects the Step-3 rules (stamps).
template <class T, int BX, int BY, int BZ, bool remedy, int GTM = kGroupThreads>
__device__ void group_pass(const FwdParams<T> &P, T *smbase, GroupCtl *gcs, GroupQueue *gqs, int it, int n,
                           unsigned kmin_cur, float width, int chunk, int *s_visits, long long &st_tiles,
                           long long &st_sweeps, long long &st_def) {
    using G = TileGeom<BX, BY, BZ>;
    using GG = GroupGeom<BX, BY, BZ, GTM>;
    Ctl *ctl = P.ctl;
    const int nslot = (it + 1) % 3;
    const int *in = (it & 1) ? P.list1 : P.list0;
    int *out = (it & 1) ? P.list0 : P.list1;
    unsigned *kcur = P.tkey + (size_t)(it & 1) * P.n_tiles;
    unsigned *knext = P.tkey + (size_t)((it + 1) & 1) * P.n_tiles;
    int *cnt_next = remedy ? &ctl->rcnt[nslot] : &ctl->cnt[nslot];
    unsigned *kmin_next = remedy ? &ctl->rkmin[nslot] : &ctl->kmin[nslot];
    int *grab = remedy ? &ctl->rgrab[it % 3] : &ctl->grab[it % 3];
    const int next_stamp = it + 2;
    const int tid = threadIdx.x;
    const int gi = tid / GG::GT, gt = tid % GG::GT, bid = 1 + gi;
    T *sm = smbase + (size_t)gi * G::S;
    GroupCtl &gc = gcs[gi];
    GroupQueue &q = gqs[gi];
    const OrderCtx ord = order_begin(remedy ? P.ordered : P.ordered_update, kmin_cur, width);
    n = min(n, P.n_tiles);
    chunk = max(1, min(chunk, GG::GT));
    const int cta_groups = blockDim.x / GG::GT;
    // the static first chunks cover the list: no grab from the shared counter
    const bool static_only = (long long)gridDim.x * cta_groups * chunk >= n;
    for (bool first = true;; first = false) {
        if (!first && static_only) break;
        if (gt == 0) {
            q.n = 0;
            q.base = grab_chunk(grab, first, blockIdx.x * cta_groups + gi, gridDim.x * cta_groups, chunk);
        }
        group_sync(bid, GG::GT);
        const int base = q.base;
        if (base >= n) break;                          // group-uniform
        // classify: one entry per thread (every lane of the group's warps takes part in the pushes);
        // the tile record is loaded beside the key, for the first queued tiles
        {
            const int e = base + gt;
            bool valid = gt < chunk && e < n;
            const int g = valid ? __ldcg(in + e) : -1;
            if (valid && dbg_bad_tile(ctl, g, P.n_tiles)) valid = false;
            unsigned key = kKeyInf;
            int4 r0 = make_int4(0, 0, 0, 0), r1 = r0;
            if (valid) {
                r0 = __ldcg(reinterpret_cast<const int4 *>(P.tile_nb + 8 * g));
                r1 = __ldcg(reinterpret_cast<const int4 *>(P.tile_nb + 8 * g + 4));
            }
            if (valid && ord.on) {
                key = __ldcg(kcur + g);
                __stcg(kcur + g, kKeyInf);               // no one writes this parity in this iteration
            }
            const bool defer = valid && ord.on && !order_visit(ord, key);
            bool want = false;
            if (defer) {
                atomicMin(knext + g, key);
                want = remedy ? atomicExch(P.tstamp + g, next_stamp) != next_stamp : true;
                st_def++;
            }
            warp_push(ctl, cnt_next, out, P.n_tiles, want, g, ord.on ? kmin_next : nullptr, key);
            if (valid && !defer) {
                const int pos = atomicAdd(&q.n, 1);
                q.tile[pos] = g;
                q.key[pos] = key;
                if (pos < kQueueRec) { q.rec[pos][0] = r0; q.rec[pos][1] = r1; }
            }
        }
        group_sync(bid, GG::GT);
        const int qn = q.n;
        // visit
        for (int qi = 0; qi < qn; ++qi) {
            if (gt == 0) {
                if (qi < kQueueRec) group_set(gc, q.tile[qi], q.key[qi], q.rec[qi][0], q.rec[qi][1]);
                else group_fetch(P, gc, q.tile[qi], q.key[qi]);
            }
            group_sync(bid, GG::GT);
            visit_and_list<T, BX, BY, BZ, remedy, GTM>(P, sm, gc, gt, bid, ord, knext, out, cnt_next, kmin_next,
                                                       next_stamp, s_visits, st_tiles, st_sweeps);
        }
    }
}

// Warp-aggregated append of kept tiles to the visit list of a two-phase
// iteration, each with its key and record (every lane of the warp calls it).
__device__ __forceinline__ void push_visit(Ctl *ctl, int *vcnt, VisitRec *vlist, int cap, bool keep, int g,
                                           unsigned key, int4 r0, int4 r1) {
    const unsigned m = __ballot_sync(kFull, keep);
    if (!m) return;
    const int lane = lane_id(), leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(vcnt, __popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (!keep) return;
    const int pos = base + __popc(m & ((1u << lane) - 1));
    if (pos < cap) {
        VisitRec *vr = vlist + pos;
        __stcg(&vr->head, make_int4(g, (int)key, 0, 0));
        __stcg(&vr->r0, r0);
        __stcg(&vr->r1, r1);
    } else {
        atomicOr(&ctl->flags, kFlagOverflow);
    }
}

// An iteration of the latency-only kernel with more visits expected than
// thread groups.  On a bucketed list it runs in two phases split by a grid
// barrier: first every thread of the launch classifies list entries (a
// deferred entry is listed again on the spot, a kept one is appended to the
// visit list); then the thread groups take the kept tiles one at a time (the
// first by group index, the others from a shared counter).  On an unordered
// list every entry is kept, so the groups take the list entries themselves,
// with no classification and no grid barrier (measured on B300: 512^3 maze
// 18.5 -> 17.9 ms, 16-shot tomography forward 6.1 -> 5.6 ms).  Taking chunks
// of the list with the visits they hold (group_pass) leaves some groups with
// several long visits while others idle: measured on the 256^3 oscillating
// workload, the slowest group of a Step-3 iteration made 3.8 visits against
// 2.3 on average and the iteration lasted twice the median group's time.
// Returns false if the grid barrier timed out.
template <class T, int BX, int BY, int BZ, bool remedy, int GTM>
__device__ bool group_pass_split(const FwdParams<T> &P, T *smbase, GroupCtl *gcs, int it, int n, unsigned kmin_cur,
                                 float width, int *s_visits, long long &st_tiles, long long &st_sweeps,
                                 long long &st_def, unsigned long long &target) {
    using G = TileGeom<BX, BY, BZ>;
    using GG = GroupGeom<BX, BY, BZ, GTM>;
    Ctl *ctl = P.ctl;
    const int slot = it % 3, nslot = (it + 1) % 3;
    const int *in = (it & 1) ? P.list1 : P.list0;
    int *out = (it & 1) ? P.list0 : P.list1;
    unsigned *kcur = P.tkey + (size_t)(it & 1) * P.n_tiles;
    unsigned *knext = P.tkey + (size_t)((it + 1) & 1) * P.n_tiles;
    int *cnt_next = remedy ? &ctl->rcnt[nslot] : &ctl->cnt[nslot];
    unsigned *kmin_next = remedy ? &ctl->rkmin[nslot] : &ctl->kmin[nslot];
    int *vcnt = remedy ? &ctl->rvcnt[slot] : &ctl->vcnt[slot];
    int *vgrab = remedy ? &ctl->rvgrab[slot] : &ctl->vgrab[slot];
    const int next_stamp = it + 2;
    const OrderCtx ord = order_begin(remedy ? P.ordered : P.ordered_update, kmin_cur, width);
    n = min(n, P.n_tiles);
    // An unordered list keeps every entry (its entries are distinct: Step-2 lists by tile state,
    // Step-3 lists by stamp): the groups take the entries themselves, with no classification, no
    // visit list and no grid barrier before the visits.
    const bool direct = !ord.on;
    // classify: a warp takes 32 consecutive entries (warp-uniform loop, every lane takes part in the
    // pushes); a kept tile goes to the visit list with its key and record
    const int lane = lane_id();
    const int nthreads = gridDim.x * blockDim.x;
    for (int e0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); !direct && e0 < n; e0 += nthreads) {
        const int e = e0 + lane;
        bool valid = e < n;
        const int g = valid ? __ldcg(in + e) : -1;
        if (valid && dbg_bad_tile(ctl, g, P.n_tiles)) valid = false;
        unsigned key = kKeyInf;
        int4 r0 = make_int4(0, 0, 0, 0), r1 = r0;
        if (valid) {
            r0 = __ldcg(reinterpret_cast<const int4 *>(P.tile_nb + 8 * g));
            r1 = __ldcg(reinterpret_cast<const int4 *>(P.tile_nb + 8 * g + 4));
        }
        if (valid && ord.on) {
            key = __ldcg(kcur + g);
            __stcg(kcur + g, kKeyInf);                 // no one writes this parity in this iteration
        }
        const bool defer = valid && ord.on && !order_visit(ord, key);
        bool want = false;
        if (defer) {
            atomicMin(knext + g, key);
            want = remedy ? atomicExch(P.tstamp + g, next_stamp) != next_stamp : true;
            st_def++;
        }
        warp_push(ctl, cnt_next, out, P.n_tiles, want, g, ord.on ? kmin_next : nullptr, key);
        push_visit(ctl, vcnt, P.vlist, P.n_tiles, valid && !defer, g, key, r0, r1);
    }
    if (!direct && !grid_sync(ctl, target, P.wait_ns)) return false;
    // visit the kept tiles
    const int tid = threadIdx.x;
    const int gi = tid / GG::GT, gt = tid % GG::GT, bid = 1 + gi;
    T *sm = smbase + (size_t)gi * G::S;
    GroupCtl &gc = gcs[gi];
    const int cta_groups = blockDim.x / GG::GT;
    const int groups = gridDim.x * cta_groups;
    const int nv = direct ? n : min(ld_volatile(vcnt), P.n_tiles);
    for (bool first = true;; first = false) {
        if (gt == 0) {
            const int idx = first ? blockIdx.x * cta_groups + gi : groups + atomicAdd(vgrab, 1);
            if (idx < nv && direct) {
                const int g = __ldcg(in + idx);
                if (dbg_bad_tile(ctl, g, P.n_tiles)) gc.tile = -1;
                else group_fetch(P, gc, g, kKeyInf);
            } else if (idx < nv) {
                const VisitRec *vr = P.vlist + idx;
                const int4 h = __ldcg(&vr->head);
                group_set(gc, h.x, (unsigned)h.y, __ldcg(&vr->r0), __ldcg(&vr->r1));
                if (dbg_bad_tile(ctl, h.x, P.n_tiles)) gc.tile = -1;
            } else {
                gc.tile = -1;
            }
        }
        group_sync(bid, GG::GT);
        if (gc.tile < 0) break;                        // group-uniform
        visit_and_list<T, BX, BY, BZ, remedy, GTM>(P, sm, gc, gt, bid, ord, knext, out, cnt_next, kmin_next,
                                                   next_stamp, s_visits, st_tiles, st_sweeps);
    }
    return true;
}

template <class T, int BX, int BY, int BZ, int GTM = kGroupThreads>
__device__ void update_pass_group(const FwdParams<T> &P, T *smbase, GroupCtl *gcs, GroupQueue *gqs, int it, int n,
                                  unsigned kmin_cur, float width, int chunk, int *s_visits, long long &st_tiles,
                                  long long &st_sweeps, long long &st_def) {
    group_pass<T, BX, BY, BZ, false, GTM>(P, smbase, gcs, gqs, it, n, kmin_cur, width, chunk, s_visits, st_tiles,
                                     st_sweeps, st_def);
}

template <class T, int BX, int BY, int BZ, int GTM = kGroupThreads>
__device__ void remedy_pass_group(const FwdParams<T> &P, T *smbase, GroupCtl *gcs, GroupQueue *gqs, int r, int n,
                                  unsigned kmin_cur, float width, int chunk, int *s_visits, long long &st_tiles,
                                  long long &st_sweeps, long long &st_def) {
    group_pass<T, BX, BY, BZ, true, GTM>(P, smbase, gcs, gqs, r, n, kmin_cur, width, chunk, s_visits, st_tiles,
                                    st_sweeps, st_def);
}

}  // namespace eik
