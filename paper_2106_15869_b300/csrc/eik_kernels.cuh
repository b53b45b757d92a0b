// eik_kernels.cuh -- the kernels of the forward solve: descriptor upload,
// Step 1 (k_init, k_sources), the Step-2/3 loops (one cooperative persistent
// launch, or one launch per iteration), and the output unpack.  Each
// iteration of a loop runs in latency mode (a thread group per tile,
// eik_group.cuh) when its list is short and in throughput mode (a warp per
// tile, eik_forward.cuh) otherwise.
#pragma once

#include <cstddef>

#include "eik_forward.cuh"
#include "eik_group.cuh"

namespace eik {

// latency mode when the list holds at most this many entries per thread group
// (deferred entries are classified by all threads of a CTA, so they are cheap)
constexpr int kGroupModeFactor = 8;

// Optional per-iteration trace of the persistent schedule (eik_set_trace):
// records of 4 x u64 = {globaltimer ns, phase (1 Step 2, 2 Step-3 seed, 3
// remedy, 4 FIM loop; plus kTraceThroughput when the iteration ran in
// throughput mode, a warp per tile), list size, tiles visited}, written by
// thread 0 of CTA 0 after the barrier that ends each iteration.
constexpr unsigned long long kTraceThroughput = 256;
__device__ unsigned long long *g_trace_buf = nullptr;
__device__ long long g_trace_cap = 0;

__device__ __forceinline__ void trace_record(long long &k, unsigned long long phase, long long n, long long visited) {
    unsigned long long *buf = g_trace_buf;
    if (buf && blockIdx.x == 0 && threadIdx.x == 0) {
        if (k < g_trace_cap) {
            unsigned long long *r = buf + 1 + 4 * k;
            r[0] = globaltimer();
            r[1] = phase;
            r[2] = (unsigned long long)n;
            r[3] = (unsigned long long)visited;
            buf[0] = (unsigned long long)(k + 1);   // record count
        }
        ++k;
    }
}

// ---------------------------------------------------------------- kernels
// Descriptor upload (by-value parameter, so that the call can be captured).
__global__ void k_write_desc(InstDesc *desc, DescChunk chunk) {
    const int i = threadIdx.x;
    if (i < chunk.count) desc[chunk.first + i] = chunk.d[i];
}

// 1/delta per instance for the ordered schedule: delta = order * (mean tile
// edge) * h * (mean slowness 1/F over passable nodes), `order` times the mean
// time to cross a tile.  The mean slowness, not one over the mean speed: in a
// medium of fast cells and slow walls (the maze: F = 1 and 1e-3) it follows
// the walls, whose crossing times set the spread of the keys; with 1/mean(F)
// the buckets were a few hundred times narrower there and an ordered solve of
// the 512^3 maze took 4x the iterations.

constexpr int kScaleThreads = 256;
constexpr int kScaleUnroll = 8;      // independent loads in flight per thread

// CTAs per instance of k_scale: many for few (large) instances, one for many
__host__ __device__ constexpr int scale_chunks(long long B) { return B <= 64 ? 64 : (B <= 4096 ? 8 : 1); }

// `chunks` CTAs per instance each reduce a slice of its per-tile statistics
// into part[]; the last CTA of the instance to finish (counted in done[],
// zeroed by k_init) combines the slices and writes the key scale.
template <int BX, int BY, int BZ>
__global__ void __launch_bounds__(kScaleThreads) k_scale(const InstDesc *desc, const float2 *tile_fstat,
                                                         float *inst_scale, int B, int chunks, float order,
                                                         ScalePart *part, int *done) {
    const int b = blockIdx.x / chunks, c = blockIdx.x % chunks;
    if (b >= B) return;
    const InstDesc &d = desc[b];
    const long long nt = (long long)d.tx * d.ty * d.tz;
    const long long per = (nt + chunks - 1) / chunks;
    const long long t_end = min(nt, (c + 1) * per);
    double sum = 0.0, cnt = 0.0;
    for (long long t0 = c * per + threadIdx.x; t0 < t_end; t0 += (long long)kScaleThreads * kScaleUnroll) {
        float2 v[kScaleUnroll];
#pragma unroll
        for (int u = 0; u < kScaleUnroll; ++u) {
            const long long t = t0 + (long long)u * kScaleThreads;
            v[u] = t < t_end ? __ldg(tile_fstat + d.tile_base + t) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kScaleUnroll; ++u) {
            sum += v[u].x; cnt += v[u].y;
        }
    }
    __shared__ double s_sum[kScaleThreads / 32], s_cnt[kScaleThreads / 32];
    __shared__ int s_last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_sum[w] = sum; s_cnt[w] = cnt; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < kScaleThreads / 32; ++q) {
            sum += s_sum[q]; cnt += s_cnt[q];
        }
        ScalePart &p = part[(size_t)b * chunks + c];
        p.sum = sum; p.cnt = cnt;
        __threadfence();
        s_last = atomicAdd(done + b, 1) == chunks - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    sum = 0.0; cnt = 0.0;
    for (int q = 0; q < chunks; ++q) {
        const ScalePart &p = part[(size_t)b * chunks + q];
        sum += ld_volatile_d(&p.sum); cnt += ld_volatile_d(&p.cnt);
    }
    const double edge = BZ == 1 ? 0.5 * (BX + BY) : (BX + BY + BZ) / 3.0;
    const double mean_slow = cnt > 0 ? sum / cnt : 0.0;
    double sc = mean_slow > 0 ? 1.0 / ((double)order * edge * d.h * mean_slow) : 1.0;
    if (!(sc > 0) || !(sc < 1e30)) sc = 1.0;
    inst_scale[b] = (float)sc;
}

// Geometry of kSpan consecutive tiles for the streaming kernels (layout
// conversion in and out of the bricks): thread t < kSpan of a CTA fills entry
// t; every thread then maps its nodes with inside() / at().
constexpr int kSpan = 4;
constexpr int kSpanThreads = 256;

template <int BX, int BY, int BZ>
struct TileSpan {
    int inst[kSpan], l[kSpan], tc[kSpan][3], lim[kSpan][3], nx[kSpan];
    long long corner[kSpan], plane[kSpan];   // node (0, 0, 0) of the tile within its instance's grid
    long long in_off[kSpan], out_off[kSpan]; // the instance's input and output offsets (no descriptor
    double h[kSpan];                         // read per element), and its spacing
    // acc: g counts the tiles of the adjoint's gradient blocks (acc_base) instead of all tiles
    __device__ void fill(const InstDesc *desc, int B, long long n_tiles, long long g0, int t, bool acc = false) {
        const long long g = g0 + t;
        int b = 0, ll = 0, tx = 0, ty = 0, tz = 0, lx = 0, ly = 0, lz = 0, nxx = 0;
        long long c = 0, pl = 0, io = 0, oo = 0;
        double hh = 0.0;
        if (g < n_tiles) {
            b = B == 1 ? 0 : acc ? find_inst_by_acc(desc, B, g) : find_inst_by_tile(desc, B, g);
            const InstDesc &d = desc[b];
            ll = (int)(g - (acc ? d.acc_base : d.tile_base));   // fewer than 2^31 tiles
            tx = ll % d.tx; ty = (ll / d.tx) % d.ty; tz = ll / (d.tx * d.ty);
            lx = min(BX, d.nx - tx * BX); ly = min(BY, d.ny - ty * BY); lz = min(BZ, d.nz - tz * BZ);
            nxx = d.nx;
            pl = (long long)d.nx * d.ny;
            c = (long long)tz * BZ * pl + (long long)ty * BY * d.nx + (long long)tx * BX;
            io = d.in_off;
            oo = d.out_off;
            hh = d.h;
        }
        inst[t] = b; l[t] = ll;
        in_off[t] = io; out_off[t] = oo; h[t] = hh;
        tc[t][0] = tx; tc[t][1] = ty; tc[t][2] = tz;
        lim[t][0] = lx; lim[t][1] = ly; lim[t][2] = lz;
        nx[t] = nxx; plane[t] = pl; corner[t] = c;
    }
    __device__ bool inside(int t, int x, int y, int z) const { return x < lim[t][0] && y < lim[t][1] && z < lim[t][2]; }
    __device__ long long at(int t, int x, int y, int z) const {
        return corner[t] + (long long)z * plane[t] + (long long)y * nx[t] + x;
    }
};

// Step 1a: bricked tau = h/F and phi = +inf; per-tile state, neighbour ids
// and (ordered schedule) slowness statistics; control block.  A CTA takes kSpan
// consecutive tiles at a time: every thread loads its kSpan * V /
// kSpanThreads speeds at once (rows of BX nodes of the caller's grid), then
// writes the bricks (one contiguous block).
template <class T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(kSpanThreads) k_init(FwdParams<T> P) {
    using G = TileGeom<BX, BY, BZ>;
    constexpr int PER = kSpan * G::V / kSpanThreads;
    static_assert(kSpan * G::V % kSpanThreads == 0 && G::V % 32 == 0, "whole nodes per thread, whole warps per tile");
    __shared__ TileSpan<BX, BY, BZ> sp;
    __shared__ float s_acc[kSpan][2];          // sum of the slownesses 1/F, count (passable nodes)
    const int tid = threadIdx.x;
    const long long total = (long long)P.n_tiles * G::V;
    for (long long g0 = (long long)blockIdx.x * kSpan; g0 < P.n_tiles; g0 += (long long)gridDim.x * kSpan) {
        if (tid < kSpan) {
            sp.fill(P.desc, P.B, P.n_tiles, g0, tid);
            s_acc[tid][0] = 0.0f; s_acc[tid][1] = 0.0f;
        }
        __syncthreads();
        T f[PER];
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int r = tid + m * kSpanThreads, t = r / G::V, q = r % G::V;
            const int x = q % BX, y = (q / BX) % BY, z = q / (BX * BY);
            f[m] = T(0);                                    // outside the grid: tau = +inf
            if (sp.inside(t, x, y, z)) f[m] = P.F[sp.in_off[t] + sp.at(t, x, y, z)];
        }
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int r = tid + m * kSpanThreads, t = r / G::V;
            const long long e = g0 * G::V + r;
            const bool pass = f[m] > T(0);
            if (e < total) {
                P.tau_t[e] = pass ? T(sp.h[t]) / f[m] : Num<T>::inf();
                P.phi_t[e] = Num<T>::inf();
            }
            if (P.ordered) {   // a warp's 32 nodes lie in one tile
                float fs = pass ? 1.0f / (float)f[m] : 0.0f;
                const int fc = __popc(__ballot_sync(0xffffffffu, pass));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) fs += __shfl_xor_sync(0xffffffffu, fs, o);
                if ((tid & 31) == 0 && fc) {
                    atomicAdd(&s_acc[t][0], fs);
                    atomicAdd(&s_acc[t][1], (float)fc);
                }
            }
        }
        __syncthreads();
        if (tid < kSpan && g0 + tid < P.n_tiles) {
            const long long g = g0 + tid;
            const int b = sp.inst[tid];
            if (sp.l[tid] == 0) P.scale_done[b] = 0;       // k_scale's completion count of this instance
            P.tile_inst[g] = b;
            P.tstate[g] = kDistant;
            P.tstamp[g] = 0;
            P.tkey[g] = kKeyInf;
            P.tkey[P.n_tiles + g] = kKeyInf;
            if (P.ordered) reinterpret_cast<float2 *>(P.tile_fstat)[g] = make_float2(s_acc[tid][0], s_acc[tid][1]);
        }
        if (tid < 8 * kSpan && g0 + tid / 8 < P.n_tiles) {   // tile records: neighbours, instance, key scale
            const int t = tid / 8, k = tid % 8;
            const int g = (int)(g0 + t);
            const InstDesc &d = P.desc[sp.inst[t]];
            const int tx = sp.tc[t][0], ty = sp.tc[t][1], tz = sp.tc[t][2];
            int nb;
            switch (k) {
                case 0: nb = tx > 0 ? g - 1 : -1; break;
                case 1: nb = tx + 1 < d.tx ? g + 1 : -1; break;
                case 2: nb = ty > 0 ? g - d.tx : -1; break;
                case 3: nb = ty + 1 < d.ty ? g + d.tx : -1; break;
                case 4: nb = tz > 0 ? g - d.tx * d.ty : -1; break;
                case 5: nb = tz + 1 < d.tz ? g + d.tx * d.ty : -1; break;
                case 6: nb = sp.inst[t]; break;
                default: nb = __float_as_int(1.0f); break;   // key scale, set by k_tile_scale
            }
            P.tile_nb[8 * (long long)g + k] = nb;
        }
        if (g0 == 0 && tid < (int)(sizeof(Ctl) / sizeof(int))) {
            const int k0 = (int)(offsetof(Ctl, kmin) / sizeof(int)), k1 = (int)(offsetof(Ctl, rkmin) / sizeof(int)) + 3;
            reinterpret_cast<unsigned *>(P.ctl)[tid] = (tid >= k0 && tid < k1) ? kKeyInf : 0u;
        }
        __syncthreads();                                       // the span is refilled next
    }
}

// the instance key scale into every tile record (ordered schedule)
__global__ void k_tile_scale(int *tile_nb, const float *inst_scale, int n_tiles) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n_tiles; g += gridDim.x * blockDim.x)
        tile_nb[8 * g + 7] = __float_as_int(inst_scale[tile_nb[8 * g + 6]]);
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

// Step 1b: sources fixed (phi = value, tau = +inf: never lowered); Active = the tiles
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
    P.tau_t[(size_t)g * G::V + loc] = Num<T>::inf();
    int cand[7];
    int nc = 0;
    cand[nc++] = g;
    if (i % BX == 0 && i > 0) cand[nc++] = g - 1;
    if (i % BX == BX - 1 && i + 1 < d.nx) cand[nc++] = g + 1;
    if (j % BY == 0 && j > 0) cand[nc++] = g - d.tx;
    if (j % BY == BY - 1 && j + 1 < d.ny) cand[nc++] = g + d.tx;
    if (k % BZ == 0 && k > 0) cand[nc++] = g - d.tx * d.ty;
    if (k % BZ == BZ - 1 && k + 1 < d.nz) cand[nc++] = g + d.tx * d.ty;
    const unsigned key = scaled_key((float)P.src_val[s], P.inst_scale[b]);
    // the first list of the loop that runs first: Step 2, or the one loop of the FIM
    int *cnt0 = P.fim ? &P.ctl->rcnt[0] : &P.ctl->cnt[0];
    unsigned *kmin0 = P.fim ? &P.ctl->rkmin[0] : &P.ctl->kmin[0];
    for (int q = 0; q < nc; ++q) {
        if (P.ordered) {
            atomicMin(P.tkey + cand[q], key);
            atomicMin(kmin0, key);
        }
        if (atomicCAS(P.tstate + cand[q], (int)kDistant, (int)kActive) == (int)kDistant) {
            const int pos = atomicAdd(cnt0, 1);
            if (pos < P.n_tiles) P.list0[pos] = cand[q];
            else atomicOr(&P.ctl->flags, kFlagOverflow);
        }
    }
}

// Statistics of one thread, summed over its warp, added to the control block.
template <class T>
__device__ __forceinline__ void flush_stats(const FwdParams<T> &P, long long a, long long b, long long c,
                                            long long d, long long e) {
    unsigned long long v[5] = {(unsigned long long)a, (unsigned long long)b, (unsigned long long)c,
                               (unsigned long long)d, (unsigned long long)e};
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if (lane_id() == 0) {
        if (v[4]) atomicAdd((unsigned long long *)&P.ctl->tiles_deferred, v[4]);
        if (v[0]) atomicAdd((unsigned long long *)&P.ctl->tiles_update, v[0]);
        if (v[1]) atomicAdd((unsigned long long *)&P.ctl->tiles_flagged, v[1]);
        if (v[2]) atomicAdd((unsigned long long *)&P.ctl->tiles_remedy, v[2]);
        if (v[3]) atomicAdd((unsigned long long *)&P.ctl->sweeps, v[3]);
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

// Persistent-kernel variants.  kPersistMixed takes each iteration in the
// latency mode or the throughput mode by its list size; kPersistLatency takes
// every iteration in the latency mode, with 256-thread groups, or 128-thread
// groups when more visits are expected than there are 256-thread groups.
// Without the throughput mode's per-lane node arrays it needs fewer
// registers, so more CTAs (and thread groups) are resident.  The host takes
// it for FP32 8x8x8 tiles, where it is faster on every workload measured
// (256^3 to 512^3 grids, ordered and unordered lists, batches of 16 and 64);
// on the other tile shapes its higher CTA count spills registers.
enum : int { kPersistMixed = 0, kPersistLatency = 1 };

template <class T, int BX, int BY, int BZ, int MODE>
constexpr int persistent_min_ctas() {
    return (MODE == kPersistLatency && sizeof(T) == 4 && min_ctas<T, BX, BY, BZ>() < 3) ? 3
                                                                                        : min_ctas<T, BX, BY, BZ>();
}

template <class T, int BX, int BY, int BZ>
struct WarpSmem {
    T phi[kWarpsPerCta][TileGeom<BX, BY, BZ>::S];
};

// Steps 2 and 3 in one cooperative launch; iterations are separated by the
// bounded grid barrier.  Every warp reads the same list size after a
// barrier, so all CTAs leave the loops together.
template <class T, int BX, int BY, int BZ, int MODE>
__global__ void __launch_bounds__(32 * kWarpsPerCta, (persistent_min_ctas<T, BX, BY, BZ, MODE>()))
    k_persistent(FwdParams<T> P) {
    using GGS = GroupGeom<BX, BY, BZ, kSmallGroupThreads>;
    using GGC = GroupGeom<BX, BY, BZ, kColumnGroupThreads>;
    constexpr int NG1 = GroupGeom<BX, BY, BZ>::NG;
    constexpr int NGS = GGS::NG > NG1 ? GGS::NG : NG1;
    constexpr int NGMAX = MODE == kPersistLatency && GGC::NG > NGS ? GGC::NG : NGS;
    __shared__ WarpSmem<T, BX, BY, BZ> sm;
    __shared__ GroupCtl gcs[NGMAX];
    __shared__ GroupQueue gqs[NG1];                    // only the chunked passes of kGroupThreads groups queue
    __shared__ int s_n, s_p, s_visits;
    __shared__ unsigned s_k;
    T *my = sm.phi[warp_in_cta()];
    init_stage<T, BX, BY, BZ>(my);
    halo_table_fill<BX, BY, BZ>();                     // read after the loop's first CTA barrier
    if (threadIdx.x == 0) s_visits = 0;
    const int groups = gridDim.x * GroupGeom<BX, BY, BZ>::NG;
    float width = 1.0f;
    int n_prev = 0;
    long long tk = 0;
    trace_record(tk, 0, 0, 0);
    Ctl *ctl = P.ctl;
    unsigned long long target = 0;
    long long t_upd = 0, t_flag = 0, t_rem = 0, sweeps = 0, deferred = 0;
    int it = 0, r = 0;
    if (P.fim) goto neighbour_check;                   // FIM: one loop, entered with the source tiles listed
    for (;; ++it) {
        if (threadIdx.x == 0) {
            s_n = ld_volatile(&ctl->cnt[it % 3]);
            s_k = ld_volatile_u(&ctl->kmin[it % 3]);
            s_p = it > 0 ? ld_volatile(&ctl->nproc[(it - 1) % 4]) : 0;
        }
        __syncthreads();
        const int n = s_n;
        const unsigned kq = s_k;
        if (it > 0) width = adapt_window(width, s_p, n_prev, groups, (int)gridDim.x * kWarpsPerCta);
        const int chunk = group_chunk(n, it > 0 ? s_p : 0, it > 0 ? n_prev : 0, groups, GroupGeom<BX, BY, BZ>::GT);
        n_prev = n;
        if (n == 0) break;
        if (it >= P.max_iters) { if (threadIdx.x == 0) atomicOr(&ctl->flags, kFlagCap); goto done; }
        if (blockIdx.x == 0 && threadIdx.x == 0) {   // slot (it+2)%3 was last read in iteration it-1
            ctl->cnt[(it + 2) % 3] = 0;
            ctl->kmin[(it + 2) % 3] = kKeyInf;
            ctl->grab[(it + 2) % 3] = 0;
            ctl->vcnt[(it + 2) % 3] = 0;
            ctl->vgrab[(it + 2) % 3] = 0;
            ctl->nproc[(it + 2) % 4] = 0;
        }
        bool thr = false;                              // this iteration in throughput mode
        if constexpr (MODE == kPersistLatency) {
            // more visits expected (the last iteration's, or the list) than groups: smaller
            // groups, one visit per grab (a bucketed list is classified first, in a phase of
            // its own)
            const int expv = it > 0 ? s_p : n;
            if (GGC::NG > GGS::NG && expv > kColumnGroupFactor * groups) {
                if (!group_pass_split<T, BX, BY, BZ, false, kColumnGroupThreads>(
                        P, &sm.phi[0][0], gcs, it, n, kq, width, &s_visits, t_upd, sweeps, deferred, target))
                    goto done;
            } else if (GGS::NG > NG1 && expv > groups) {
                if (!group_pass_split<T, BX, BY, BZ, false, kSmallGroupThreads>(
                        P, &sm.phi[0][0], gcs, it, n, kq, width, &s_visits, t_upd, sweeps, deferred, target))
                    goto done;
            } else
                update_pass_group<T, BX, BY, BZ>(P, &sm.phi[0][0], gcs, gqs, it, n, kq, width, chunk, &s_visits,
                                                 t_upd, sweeps, deferred);
        } else if (n <= kGroupModeFactor * groups) {
            update_pass_group<T, BX, BY, BZ>(P, &sm.phi[0][0], gcs, gqs, it, n, kq, width, chunk, &s_visits, t_upd,
                                             sweeps, deferred);
        } else {
            thr = true;
            update_pass<T, BX, BY, BZ>(P, my, it, n, kq, width, &s_visits, t_upd, sweeps, deferred);
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_visits) { atomicAdd(&ctl->nproc[it % 4], s_visits); s_visits = 0; }
        if (!grid_sync(ctl, target, P.wait_ns)) goto done;
        trace_record(tk, 1 | (thr ? kTraceThroughput : 0), n, ld_volatile(&ctl->nproc[it % 4]));
    }
    if (P.skip_remedy) goto done;
    detect_pass<T, BX, BY, BZ>(P, my, t_flag);
    if (!grid_sync(ctl, target, P.wait_ns)) goto done;
    trace_record(tk, 2, P.n_tiles, ld_volatile(&ctl->rcnt[0]));
    // the Step-2 counters are idle from here on: nproc slots restart for Step 3
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) ctl->nproc[q] = 0;
    if (!grid_sync(ctl, target, P.wait_ns)) goto done;
neighbour_check:
    // Step 3b; under the FIM the whole solve.  A visit lists the neighbour
    // tiles across the faces where its values dropped, whatever their state.
    width = 1.0f;
    n_prev = 0;
    for (;; ++r) {
        if (threadIdx.x == 0) {
            s_n = ld_volatile(&ctl->rcnt[r % 3]);
            s_k = ld_volatile_u(&ctl->rkmin[r % 3]);
            s_p = r > 0 ? ld_volatile(&ctl->nproc[(r - 1) % 4]) : 0;
        }
        __syncthreads();
        const int n = s_n;
        const unsigned kq = s_k;
        if (r > 0) width = adapt_window(width, s_p, n_prev, groups, (int)gridDim.x * kWarpsPerCta);
        const int chunk = group_chunk(n, r > 0 ? s_p : 0, r > 0 ? n_prev : 0, groups, GroupGeom<BX, BY, BZ>::GT);
        n_prev = n;
        if (n == 0) break;
        if (r >= P.max_iters) { if (threadIdx.x == 0) atomicOr(&ctl->flags, kFlagCap); goto done; }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctl->rcnt[(r + 2) % 3] = 0;
            ctl->rkmin[(r + 2) % 3] = kKeyInf;
            ctl->rgrab[(r + 2) % 3] = 0;
            ctl->rvcnt[(r + 2) % 3] = 0;
            ctl->rvgrab[(r + 2) % 3] = 0;
            ctl->nproc[(r + 2) % 4] = 0;
        }
        bool thr = false;
        if constexpr (MODE == kPersistLatency) {
            const int expv = r > 0 ? s_p : n;
            if (GGC::NG > GGS::NG && expv > kColumnGroupFactor * groups) {
                if (!group_pass_split<T, BX, BY, BZ, true, kColumnGroupThreads>(
                        P, &sm.phi[0][0], gcs, r, n, kq, width, &s_visits, t_rem, sweeps, deferred, target))
                    goto done;
            } else if (GGS::NG > NG1 && expv > groups) {
                if (!group_pass_split<T, BX, BY, BZ, true, kSmallGroupThreads>(
                        P, &sm.phi[0][0], gcs, r, n, kq, width, &s_visits, t_rem, sweeps, deferred, target))
                    goto done;
            } else
                remedy_pass_group<T, BX, BY, BZ>(P, &sm.phi[0][0], gcs, gqs, r, n, kq, width, chunk, &s_visits,
                                                 t_rem, sweeps, deferred);
        } else if (n <= kGroupModeFactor * groups) {
            remedy_pass_group<T, BX, BY, BZ>(P, &sm.phi[0][0], gcs, gqs, r, n, kq, width, chunk, &s_visits, t_rem,
                                             sweeps, deferred);
        } else {
            thr = true;
            remedy_pass<T, BX, BY, BZ>(P, my, r, n, kq, width, &s_visits, t_rem, sweeps, deferred);
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_visits) { atomicAdd(&ctl->nproc[r % 4], s_visits); s_visits = 0; }
        if (!grid_sync(ctl, target, P.wait_ns)) goto done;
        trace_record(tk, (P.fim ? 4 : 3) | (thr ? kTraceThroughput : 0), n, ld_volatile(&ctl->nproc[r % 4]));
    }
done:
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->iters_update = it;
        ctl->iters_remedy = r;
    }
    flush_stats<T>(P, t_upd, t_flag, t_rem, sweeps, deferred);
}

// Host-loop schedule: one launch per iteration.  The bucket width of
// iteration it comes from the width of it-1 (ctl->win by parity: launch it
// reads slot (it-1)&1 and its block 0 writes slot it&1) and the visits of it-1.
template <int BX, int BY, int BZ>
__device__ __forceinline__ float host_loop_width(Ctl *ctl, int it, int n, int prev_n) {
    (void)n;
    const float w_prev = it > 0 ? *(volatile float *)&ctl->win[(it - 1) & 1] : 1.0f;
    const float w = it > 0 ? adapt_window(w_prev, ld_volatile(&ctl->nproc[(it - 1) % 4]), prev_n,
                                          (int)gridDim.x * GroupGeom<BX, BY, BZ>::NG, (int)gridDim.x * kWarpsPerCta)
                           : 1.0f;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->win[it & 1] = w;
    return w;
}

// Host-loop schedule: one launch per iteration.
template <class T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(32 * kWarpsPerCta, (min_ctas<T, BX, BY, BZ>())) k_update_iter(FwdParams<T> P, int it,
                                                                                              int prev_n) {
    __shared__ WarpSmem<T, BX, BY, BZ> sm;
    __shared__ GroupCtl gcs[GroupGeom<BX, BY, BZ>::NG];
    __shared__ GroupQueue gqs[GroupGeom<BX, BY, BZ>::NG];
    __shared__ int s_visits;
    const int n = ld_volatile(&P.ctl->cnt[it % 3]);
    const unsigned kq = ld_volatile_u(&P.ctl->kmin[it % 3]);
    const float width = host_loop_width<BX, BY, BZ>(P.ctl, it, n, prev_n);
    const int groups = (int)gridDim.x * GroupGeom<BX, BY, BZ>::NG;
    const int chunk = group_chunk(n, it > 0 ? ld_volatile(&P.ctl->nproc[(it - 1) % 4]) : 0, it > 0 ? prev_n : 0, groups,
                                  GroupGeom<BX, BY, BZ>::GT);
    long long t = 0, s = 0, d = 0;
    init_stage<T, BX, BY, BZ>(sm.phi[warp_in_cta()]);
    halo_table_fill<BX, BY, BZ>();
    if (threadIdx.x == 0) s_visits = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.ctl->cnt[(it + 2) % 3] = 0;
        P.ctl->kmin[(it + 2) % 3] = kKeyInf;
        P.ctl->grab[(it + 2) % 3] = 0;
        P.ctl->nproc[(it + 2) % 4] = 0;
    }
    __syncthreads();
    if (n <= kGroupModeFactor * groups)
        update_pass_group<T, BX, BY, BZ>(P, &sm.phi[0][0], gcs, gqs, it, n, kq, width, chunk, &s_visits, t, s, d);
    else
        update_pass<T, BX, BY, BZ>(P, sm.phi[warp_in_cta()], it, n, kq, width, &s_visits, t, s, d);
    __syncthreads();
    if (threadIdx.x == 0 && s_visits) atomicAdd(&P.ctl->nproc[it % 4], s_visits);
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
__global__ void __launch_bounds__(32 * kWarpsPerCta, (min_ctas<T, BX, BY, BZ>())) k_remedy_iter(FwdParams<T> P, int r,
                                                                                              int prev_n) {
    __shared__ WarpSmem<T, BX, BY, BZ> sm;
    __shared__ GroupCtl gcs[GroupGeom<BX, BY, BZ>::NG];
    __shared__ GroupQueue gqs[GroupGeom<BX, BY, BZ>::NG];
    __shared__ int s_visits;
    const int n = ld_volatile(&P.ctl->rcnt[r % 3]);
    const unsigned kq = ld_volatile_u(&P.ctl->rkmin[r % 3]);
    const float width = host_loop_width<BX, BY, BZ>(P.ctl, r, n, prev_n);
    const int groups = (int)gridDim.x * GroupGeom<BX, BY, BZ>::NG;
    const int chunk = group_chunk(n, r > 0 ? ld_volatile(&P.ctl->nproc[(r - 1) % 4]) : 0, r > 0 ? prev_n : 0, groups,
                                  GroupGeom<BX, BY, BZ>::GT);
    long long t = 0, s = 0, d = 0;
    init_stage<T, BX, BY, BZ>(sm.phi[warp_in_cta()]);
    halo_table_fill<BX, BY, BZ>();
    if (threadIdx.x == 0) s_visits = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.ctl->rcnt[(r + 2) % 3] = 0;
        P.ctl->rkmin[(r + 2) % 3] = kKeyInf;
        P.ctl->rgrab[(r + 2) % 3] = 0;
        P.ctl->nproc[(r + 2) % 4] = 0;
    }
    __syncthreads();
    if (n <= kGroupModeFactor * groups)
        remedy_pass_group<T, BX, BY, BZ>(P, &sm.phi[0][0], gcs, gqs, r, n, kq, width, chunk, &s_visits, t, s, d);
    else
        remedy_pass<T, BX, BY, BZ>(P, sm.phi[warp_in_cta()], r, n, kq, width, &s_visits, t, s, d);
    __syncthreads();
    if (threadIdx.x == 0 && s_visits) atomicAdd(&P.ctl->nproc[r % 4], s_visits);
    flush_stats<T>(P, 0, 0, t, s, d);
}

// Output: bricked phi -> the caller's row-major phi.  A CTA takes kSpan
// consecutive bricks at a time (one contiguous block); every thread loads its
// kSpan * V / kSpanThreads nodes at once (coalesced, streaming), then stores
// them (rows of BX nodes of the caller's grid).
template <class T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(kSpanThreads) k_unpack(FwdParams<T> P) {
    using G = TileGeom<BX, BY, BZ>;
    constexpr int PER = kSpan * G::V / kSpanThreads;
    __shared__ TileSpan<BX, BY, BZ> sp;
    const long long total = (long long)P.n_tiles * G::V;
    for (long long g0 = (long long)blockIdx.x * kSpan; g0 < P.n_tiles; g0 += (long long)gridDim.x * kSpan) {
        if (threadIdx.x < kSpan) sp.fill(P.desc, P.B, P.n_tiles, g0, threadIdx.x);
        __syncthreads();
        T val[PER];
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const long long e = g0 * G::V + threadIdx.x + (long long)m * kSpanThreads;
            val[m] = e < total ? __ldcs(P.phi_t + e) : T(0);
        }
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int r = threadIdx.x + m * kSpanThreads, t = r / G::V, q = r % G::V;
            const int x = q % BX, y = (q / BX) % BY, z = q / (BX * BY);
            if (sp.inside(t, x, y, z)) P.phi_out[sp.out_off[t] + sp.at(t, x, y, z)] = val[m];
        }
        __syncthreads();                                            // the span is refilled next
    }
}

}  // namespace eik
