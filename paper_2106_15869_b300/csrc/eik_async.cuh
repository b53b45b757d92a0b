// eik_async.cuh -- the asynchronous schedule of the improved FIM (sm_103a).
//
// Same sets and rules as the iteration-synchronous schedule (Algorithm 2 at
// tile granularity), but the Active and Remedy sets are held in a device-wide
// FIFO work queue instead of per-iteration lists: a warp takes the next tile,
// visits it, and queues the tiles the rules add, with no barrier between
// visits.  A tile is never visited by two warps at once and never queued
// twice (per-tile queue state), so the only grid-wide barriers are between
// Step 2, the Step-3 recomputation and the remedy loop.  Each phase ends when
// no tile is queued or being visited (a pending counter reaching zero).  The
// fixed point reached is the same unique discrete solution.
//
// Queue: a bounded multi-producer multi-consumer ring of Q = 2^k slots with a
// sequence number per slot (position p uses slot p mod Q; the producer of p
// waits until seq == p, writes, sets seq = p + 1; the consumer of p waits
// until seq == p + 1, reads, sets seq = p + Q).  Q exceeds the number of tiles
// plus warps, so a producer never waits for a consumer that has not claimed
// its position.  Every wait is bounded by the call's wait limit (Q.wait_ns).
#pragma once

#include "eik_kernels.cuh"

namespace eik {

enum QState : int { kIdle = 0, kQueued = 1, kBusy = 2, kBusyRequeue = 3 };

struct AsyncQ {
    int *data;                    // [Q] tile ids
    unsigned long long *seq;      // [Q] slot sequence numbers
    int *qstate;                  // [n_tiles] QState
    unsigned long long mask;      // Q - 1
    long long visit_cap;          // visits allowed per phase
    unsigned long long wait_ns;   // bound on every wait of the queue
    int n_tiles;                  // tile ids in the ring lie in [0, n_tiles)
};

__device__ __forceinline__ unsigned long long ld_acq_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// one lane: append g (counted in q_pending first, so the phase cannot end
// while g is on its way into the ring)
__device__ __forceinline__ bool q_enqueue(Ctl *ctl, const AsyncQ &Q, int g) {
    atomicAdd(&ctl->q_pending, 1);
    const unsigned long long p = atomicAdd(&ctl->q_tail, 1ull);
    unsigned long long *sq = Q.seq + (p & Q.mask);
    const unsigned long long t0 = globaltimer();
    while (ld_acq_u64(sq) != p) {
        if (ld_volatile(&ctl->abort)) return false;
        if (globaltimer() - t0 > Q.wait_ns) {
            atomicOr(&ctl->flags, kFlagTimeout);
            atomicExch(&ctl->abort, 1);
            return false;
        }
        __nanosleep(32);
    }
    __stcg(Q.data + (p & Q.mask), g);
    __threadfence();
    st_release(sq, p + 1);
    return true;
}

// one lane: ask for a visit of g (queue it, or flag a re-visit if it is being visited)
__device__ __forceinline__ void q_request(Ctl *ctl, const AsyncQ &Q, int g) {
    int s = ld_volatile(Q.qstate + g);
    for (int tries = 0; tries < 64; ++tries) {
        if (s == kQueued || s == kBusyRequeue) return;
        const int want = s == kIdle ? kQueued : kBusyRequeue;
        const int prev = atomicCAS(Q.qstate + g, s, want);
        if (prev == s) {
            if (want == kQueued) q_enqueue(ctl, Q, g);
            return;
        }
        s = prev;
    }
    atomicOr(&ctl->flags, kFlagOverflow);     // cannot happen: every CAS failure moves s forward
}

// one lane: the visit of g is over; queue it again if a re-visit was asked meanwhile
__device__ __forceinline__ void q_finish(Ctl *ctl, const AsyncQ &Q, int g) {
    if (atomicCAS(Q.qstate + g, (int)kBusy, (int)kIdle) != (int)kBusy) {
        atomicExch(Q.qstate + g, (int)kQueued);
        q_enqueue(ctl, Q, g);
    }
}

// warp: take the next tile, or -1 when the phase is over (nothing queued or
// being visited, or an abort).  A position is retired (marked consumed) only
// when nothing is pending, because only then can no producer still fill it;
// after the visit cap, entries are taken and dropped until nothing is pending.
__device__ __forceinline__ int q_pop(Ctl *ctl, const AsyncQ &Q) {
    int g = -1;
    if (lane_id() == 0) {
        unsigned long long p = atomicAdd(&ctl->q_head, 1ull);
        unsigned long long t0 = globaltimer();
        for (;;) {
            unsigned long long *sq = Q.seq + (p & Q.mask);
            const unsigned long long sv = ld_acq_u64(sq);
            if (sv == p + 1) {
                const int e = __ldcg(Q.data + (p & Q.mask));
                st_release(sq, p + Q.mask + 1);
                if (dbg_bad_tile(ctl, e, Q.n_tiles)) {
                    // debug build: an entry that is not a tile id is consumed and dropped
                    atomicSub(&ctl->q_pending, 1);
                    p = atomicAdd(&ctl->q_head, 1ull);
                    t0 = globaltimer();
                    continue;
                }
                if (!ld_volatile(&ctl->q_stop)) { g = e; break; }
                // draining after the visit cap: drop the entry, claim the next position
                __stcg(Q.qstate + e, (int)kIdle);
                __threadfence();
                atomicSub(&ctl->q_pending, 1);
                p = atomicAdd(&ctl->q_head, 1ull);
                t0 = globaltimer();
                continue;
            }
            // sv == p: not filled yet; sv < p: the consumer of p - Q is still releasing
            if (sv == p && ld_volatile(&ctl->q_pending) == 0) {
                st_release(sq, p + Q.mask + 1);     // no producer can fill p in this phase
                break;
            }
            if (ld_volatile(&ctl->abort)) break;
            if (globaltimer() - t0 > Q.wait_ns) {
                atomicOr(&ctl->flags, kFlagTimeout);
                atomicExch(&ctl->abort, 1);
                break;
            }
            __nanosleep(64);
        }
        if (g >= 0) {
            __stcg(Q.qstate + g, (int)kBusy);
            if (atomicAdd((unsigned long long *)&ctl->q_visits, 1ull) >= (unsigned long long)Q.visit_cap) {
                atomicOr(&ctl->flags, kFlagCap);
                atomicExch(&ctl->q_stop, 1);
            }
        }
        __threadfence();
    }
    return __shfl_sync(kFull, g, 0);
}

__device__ __forceinline__ void q_done(Ctl *ctl) {
    if (lane_id() == 0) {
        __threadfence();
        atomicSub(&ctl->q_pending, 1);
    }
}

// Step 2, asynchronous: a visit that changes the tile asks for a re-visit
// (the tile stays Active); a visit that changes nothing moves the tile to
// Source and activates (queues) its Distant face neighbours.
template <class T, int BX, int BY, int BZ>
__device__ void async_update_phase(const FwdParams<T> &P, const AsyncQ &Q, T *sm, long long &st_tiles,
                                   long long &st_sweeps) {
    using G = TileGeom<BX, BY, BZ>;
    Ctl *ctl = P.ctl;
    const int lane = lane_id();
    for (;;) {
        const int g = q_pop(ctl, Q);
        if (g < 0) break;
        int nbf = lane < 6 ? __ldcg(P.tile_nb + 8 * g + lane) : -1;
        if ((unsigned)nbf >= (unsigned)P.n_tiles) nbf = -1;
        T v[G::NPL], tau[G::NPL];
        stage_tile<T, BX, BY, BZ>(P, sm, g, nbf, v, tau);
        unsigned mine;
        bool changed;
        const int s = relax_tile<T, BX, BY, BZ>(sm, v, tau, P.max_sweeps, P.mt, mine, changed);
        write_back<T, BX, BY, BZ>(P, g, mine, v);
        __threadfence();
        __syncwarp();
        if (lane == 0) { st_tiles++; st_sweeps += s; }
        if (changed && (!P.one_visit || s >= P.max_sweeps)) {
            if (lane == 0) q_request(ctl, Q, g);                    // stays Active
        } else {
            if (lane == 0) __stcg(P.tstate + g, (int)kSource);      // Active -> Source
            if (nbf >= 0 && atomicCAS(P.tstate + nbf, (int)kDistant, (int)kActive) == (int)kDistant)
                q_request(ctl, Q, nbf);
        }
        __syncwarp();
        if (lane == 0) q_finish(ctl, Q, g);
        q_done(ctl);
        __syncwarp();
    }
}

// Step 3b, asynchronous: a Remedy tile is relaxed (decrease only) and asks for
// visits of the neighbour tiles across the faces where its values dropped.
template <class T, int BX, int BY, int BZ>
__device__ void async_remedy_phase(const FwdParams<T> &P, const AsyncQ &Q, T *sm, long long &st_tiles,
                                   long long &st_sweeps) {
    using G = TileGeom<BX, BY, BZ>;
    Ctl *ctl = P.ctl;
    const int lane = lane_id();
    for (;;) {
        const int g = q_pop(ctl, Q);
        if (g < 0) break;
        int nbf = lane < 6 ? __ldcg(P.tile_nb + 8 * g + lane) : -1;
        if ((unsigned)nbf >= (unsigned)P.n_tiles) nbf = -1;
        T v[G::NPL], tau[G::NPL];
        stage_tile<T, BX, BY, BZ>(P, sm, g, nbf, v, tau);
        unsigned mine;
        bool changed;
        const int s = relax_tile<T, BX, BY, BZ>(sm, v, tau, P.max_sweeps, P.mt, mine, changed);
        write_back<T, BX, BY, BZ>(P, g, mine, v);
        __threadfence();
        __syncwarp();
        const int fm = lowering_faces<T, BX, BY, BZ>(mine, v, sm);
        if (lane == 0) { st_tiles++; st_sweeps += s; }
        if (lane < 6 && (fm >> lane & 1) && nbf >= 0) q_request(ctl, Q, nbf);
        if (lane == 6 && changed && s >= P.max_sweeps) q_request(ctl, Q, g);
        __syncwarp();
        if (lane == 0) q_finish(ctl, Q, g);
        q_done(ctl);
        __syncwarp();
    }
}

// Step 3a for the asynchronous schedule: recompute every tile once and queue
// the tiles holding a non-source node whose root is below its value.
template <class T, int BX, int BY, int BZ>
__device__ void async_detect_pass(const FwdParams<T> &P, const AsyncQ &Q, T *sm, long long &st_flagged) {
    using G = TileGeom<BX, BY, BZ>;
    Ctl *ctl = P.ctl;
    const int lane = lane_id();
    for (int g = warp_global(); g < P.n_tiles; g += warps_total()) {
        int nbf = lane < 6 ? __ldcg(P.tile_nb + 8 * g + lane) : -1;
        if ((unsigned)nbf >= (unsigned)P.n_tiles) nbf = -1;
        T v[G::NPL], tau[G::NPL];
        stage_tile<T, BX, BY, BZ>(P, sm, g, nbf, v, tau);
        bool low = false;
#pragma unroll
        for (int m = 0; m < G::NPL; ++m) {
            const int c = G::sidx_of(lane + 32 * m);
            const T ax = vmin(sm[c - 1], sm[c + 1]);
            const T ay = vmin(sm[c - G::SX], sm[c + G::SX]);
            const T az = vmin(sm[c - G::SX * G::SY], sm[c + G::SX * G::SY]);
            low |= node_solve(ax, ay, az, tau[m], P.mt) < v[m];
        }
        if (__any_sync(kFull, low) && lane == 0) {
            st_flagged++;
            q_request(ctl, Q, g);
        }
        __syncwarp();
    }
}

// The whole of Steps 2 and 3 in one cooperative launch: two grid barriers
// (under the FIM, its one loop and none).
template <class T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(32 * kWarpsPerCta, (min_ctas<T, BX, BY, BZ>())) k_async(FwdParams<T> P, AsyncQ Q) {
    __shared__ WarpSmem<T, BX, BY, BZ> sm;
    T *my = sm.phi[warp_in_cta()];
    init_stage<T, BX, BY, BZ>(my);
    Ctl *ctl = P.ctl;
    unsigned long long target = 0;
    long long t_upd = 0, t_flag = 0, t_rem = 0, sweeps = 0;
    if (P.fim) goto neighbour_check;                   // FIM: the queue holds the source tiles
    async_update_phase<T, BX, BY, BZ>(P, Q, my, t_upd, sweeps);
    if (!grid_sync(ctl, target, P.wait_ns)) goto done;
    if (ld_volatile(&ctl->q_stop) || P.skip_remedy) goto done;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // every claimed position was consumed or retired: restart the ring there
        const unsigned long long h = ctl->q_head;
        ctl->q_tail = h;
        ctl->q_pending = 0;
        ctl->q_visits = 0;
    }
    if (!grid_sync(ctl, target, P.wait_ns)) goto done;
    async_detect_pass<T, BX, BY, BZ>(P, Q, my, t_flag);
    if (!grid_sync(ctl, target, P.wait_ns)) goto done;
neighbour_check:
    async_remedy_phase<T, BX, BY, BZ>(P, Q, my, t_rem, sweeps);
done:
    flush_stats<T>(P, t_upd, t_flag, t_rem, sweeps, 0);
}

// Queue set-up: seq[s] = s, every tile idle.
__global__ void k_queue_init(AsyncQ Q, int n_tiles) {
    const unsigned long long n = Q.mask + 1;
    for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s < n;
         s += (unsigned long long)gridDim.x * blockDim.x) {
        Q.seq[s] = s;
        if (s < (unsigned long long)n_tiles) Q.qstate[s] = kIdle;
    }
}

// Step 1b for the asynchronous schedule: the initial tiles (listed in list0 by
// k_sources, *count of them) go into the queue.
__global__ void k_queue_seed(AsyncQ Q, Ctl *ctl, const int *count, const int *list0) {
    const int n = min(*count, (int)(Q.mask + 1));
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int g = list0[i];
        Q.qstate[g] = kQueued;
        Q.seq[i] = (unsigned long long)i + 1;
        Q.data[i] = g;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->q_tail = (unsigned long long)n;
        ctl->q_head = 0;
        ctl->q_pending = n;
    }
}

}  // namespace eik
