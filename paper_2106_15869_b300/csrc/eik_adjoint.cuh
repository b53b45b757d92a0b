// eik_adjoint.cuh -- adjoint of the discrete Eikonal solve (sm_103a).
//
// Not in the paper: the gradient of a loss L(phi) with respect to slowness
// s = 1/F, by the adjoint-state method (Leung & Qian 2006) applied to the
// residual of eq. (6) at a non-source node i,
//   G_i(phi, s) = sum_d ((phi_i - m_{i,d})^+)^2 - h^2 s_i^2 = 0,
// with m_{i,d} the selected upwind neighbour on axis d (argmin of the two
// neighbours; on a tie the lower flat index).  With w_{i,d} = 2 (phi_i -
// m_{i,d})^+ and r = dL/dphi, the adjoint lambda solves J^T lambda = r:
//   lambda_j J_jj = r_j + sum_{i : m_{i,d} = j} w_{i,d} lambda_i,
//   J_jj = sum_d w_{j,d},
// and dL/ds_j = 2 h^2 s_j lambda_j = 2 h tau_j lambda_j (tau = h/F), 0 at
// sources and at unreachable or impassable nodes.  w_{i,d} > 0 needs phi_i >
// phi_j, so the dependencies form a DAG oriented against the arrival times:
// lambda flows from the receivers back toward the sources.
//
// GPU form: the same tile machinery as the forward solve.  A listed tile is
// staged (phi with a two-node face halo, to know whether a neighbour i of j
// selects j, which needs the neighbour beyond i; lambda with a one-node
// halo), each node computes its own J_jj and the six weights w_{i->j} of its
// neighbours once, then lambda is relaxed in place by sweeps inside the tile
// until nothing changes (exact: on a DAG a value computed from final inputs is
// final, and the sum has a fixed order, so the result does not depend on the
// schedule).  Neighbour tiles across faces where lambda changed are listed.
// Sources keep lambda = 0, so they feed nothing upstream.
//
// Order: lambda_j is final once every neighbour with a larger phi is final,
// so the lists are visited by a static key per tile, -max(phi) over the tile
// in units of 1/delta (delta = order * max(phi) / (tiles along x+y+z)):
// tiles whose key lies within the window of the list's smallest key are
// visited, the others deferred, as in the forward's bucketed order (the
// result does not depend on it).
#pragma once

#include <cstddef>

#include "eik_kernels.cuh"

namespace eik {

// threads per adjoint group: 128 (four nodes per thread on 8x8x8 tiles).  The
// adjoint's visits are cheaper than the forward's and more of them run at
// once; measured on the 192^3 tomography batch, 256-thread groups are 1.2x
// slower.
constexpr int kAdjGroupThreads = 128;
template <int BX, int BY, int BZ>
using AdjGroupGeom = GroupGeom<BX, BY, BZ, kAdjGroupThreads>;

template <class T>
struct AdjParams {
    const InstDesc *desc;       // in_off: F offset; out_off: phi and r offset; aux_off: gradient offset
    int B;
    int n_tiles;
    int n_acc_tiles;            // tiles of the gradient blocks (of their first instances)
    int *tile_rec;              // [n_tiles][8]: neighbours, instance, unused
    int *tstamp;
    int *list0, *list1;
    VisitRec *vlist;            // tiles kept by the classification of a two-phase iteration
    T *phi_t, *tau_t, *lam_t, *r_t;
    Ctl *ctl;
    long long max_iters;
    int max_sweeps;
    const T *F;
    const T *phi_in;
    const T *r_in;              // dL/dphi, same offsets as phi
    const long long *src_idx;
    long long n_src;
    T *g_out;
    unsigned *tkey;             // [n_tiles] static key (ordered lists)
    float *inst_scale;          // [B] 1/delta per instance
    int ordered;
    float order;
    unsigned long long wait_ns;  // bound on every device wait of the call
};

template <int BX, int BY, int BZ>
struct AdjGeom {
    using G = TileGeom<BX, BY, BZ>;
    // phi staged with a two-node halo on every face (edges and corners unused)
    static constexpr int PX = BX + 4, PY = BY + 4, PZ = BZ + 4;
    static constexpr int PS = PX * PY * PZ;
    static __device__ __forceinline__ int pidx(int x, int y, int z) { return ((z + 2) * PY + (y + 2)) * PX + (x + 2); }
};

template <class T, int BX, int BY, int BZ>
struct AdjSmem {
    T phi[AdjGeom<BX, BY, BZ>::PS];
    T lam[TileGeom<BX, BY, BZ>::S];
};

// Step 0: bricks of tau, phi, r; lambda = 0; tile records (slot 7: the largest
// finite phi of the tile, for the list key); control block.  tstamp marks the
// tiles that seed the first list: those holding a node with r != 0 and finite
// phi (a tile whose only such nodes are sources gets one visit that changes
// nothing).  A CTA takes kSpan consecutive tiles at a time, every thread
// loading its nodes of the three input arrays at once.
template <class T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(kSpanThreads) k_adj_init(AdjParams<T> P) {
    using G = TileGeom<BX, BY, BZ>;
    constexpr int PER = kSpan * G::V / kSpanThreads;
    static_assert(kSpan * G::V % kSpanThreads == 0 && G::V % 32 == 0, "whole nodes per thread, whole warps per tile");
    __shared__ TileSpan<BX, BY, BZ> sp;
    __shared__ unsigned s_mx[kSpan];           // largest finite phi, encoded (key_enc is monotone)
    __shared__ int s_seed[kSpan];
    const int tid = threadIdx.x;
    const long long total = (long long)P.n_tiles * G::V;
    for (long long g0 = (long long)blockIdx.x * kSpan; g0 < P.n_tiles; g0 += (long long)gridDim.x * kSpan) {
        if (tid < kSpan) {
            sp.fill(P.desc, P.B, P.n_tiles, g0, tid);
            s_mx[tid] = key_enc(-__int_as_float(0x7f800000));
            s_seed[tid] = 0;
        }
        __syncthreads();
        T f[PER], ph[PER], rr[PER];
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int r = tid + m * kSpanThreads, t = r / G::V, q = r % G::V;
            const int x = q % BX, y = (q / BX) % BY, z = q / (BX * BY);
            f[m] = T(0); ph[m] = Num<T>::inf(); rr[m] = T(0);
            if (sp.inside(t, x, y, z)) {
                const long long p = sp.at(t, x, y, z);
                f[m] = P.F[sp.in_off[t] + p];
                ph[m] = P.phi_in[sp.out_off[t] + p];
                rr[m] = P.r_in[sp.out_off[t] + p];
            }
        }
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int r = tid + m * kSpanThreads, t = r / G::V;
            const long long e = g0 * G::V + r;
            const bool fin = ph[m] < Num<T>::inf();
            if (!fin) rr[m] = T(0);                                    // an unreachable receiver has no gradient
            if (e < total) {
                P.tau_t[e] = f[m] > T(0) ? T(sp.h[t]) / f[m] : Num<T>::inf();
                P.phi_t[e] = ph[m];
                P.lam_t[e] = T(0);
                P.r_t[e] = rr[m];
            }
            // a warp's 32 nodes lie in one tile
            const unsigned k = __reduce_max_sync(0xffffffffu, fin ? key_enc((float)ph[m]) : key_enc(-__int_as_float(0x7f800000)));
            const bool any = __any_sync(0xffffffffu, rr[m] != T(0));
            if ((tid & 31) == 0) {
                atomicMax(&s_mx[t], k);
                if (any) s_seed[t] = 1;
            }
        }
        __syncthreads();
        if (tid < kSpan && g0 + tid < P.n_tiles) {
            const long long g = g0 + tid;
            P.tile_rec[8 * g + 7] = __float_as_int(key_dec(s_mx[tid]));
            P.tstamp[g] = s_seed[tid];
        }
        if (tid < 8 * kSpan && tid % 8 < 7 && g0 + tid / 8 < P.n_tiles) {   // neighbours and instance
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
                default: nb = sp.inst[t]; break;
            }
            P.tile_rec[8 * (long long)g + k] = nb;
        }
        if (g0 == 0 && tid < (int)(sizeof(Ctl) / sizeof(int))) {
            const int k0 = (int)(offsetof(Ctl, kmin) / sizeof(int)), k1 = (int)(offsetof(Ctl, rkmin) / sizeof(int)) + 3;
            reinterpret_cast<unsigned *>(P.ctl)[tid] = (tid >= k0 && tid < k1) ? kKeyInf : 0u;
        }
        __syncthreads();                                       // the span is refilled next
    }
}

template <class T>
__global__ void k_adj_scale(AdjParams<T> P) {
    const int b = blockIdx.x;
    if (b >= P.B) return;
    const InstDesc &d = P.desc[b];
    const long long nt = (long long)d.tx * d.ty * d.tz;
    float mx = 0.0f;
    for (long long t = threadIdx.x; t < nt; t += blockDim.x)
        mx = fmaxf(mx, __int_as_float(P.tile_rec[8 * (d.tile_base + t) + 7]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ float s_mx[32];
    if ((threadIdx.x & 31) == 0) s_mx[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, s_mx[w]);
    const float hops = (float)(d.tx + d.ty + d.tz);
    P.inst_scale[b] = (mx > 0.0f && mx < __int_as_float(0x7f800000)) ? hops / (P.order * mx) : 0.0f;
}

// List keys (ordered lists) and the first list: the tiles k_adj_init marked.
template <class T>
__global__ void k_adj_list(AdjParams<T> P) {
    for (int g0 = blockIdx.x * blockDim.x; g0 < P.n_tiles; g0 += gridDim.x * blockDim.x) {   // uniform per warp
        const int g = g0 + (int)threadIdx.x;
        const bool valid = g < P.n_tiles;
        unsigned key = kKeyInf;
        if (valid && P.ordered) {
            const float mx = __int_as_float(P.tile_rec[8 * g + 7]);
            const float sc = P.inst_scale[P.tile_rec[8 * g + 6]];
            key = (mx > -__int_as_float(0x7f800000)) ? scaled_key(-mx, sc) : key_enc(0.0f);
            P.tkey[g] = key;
        }
        const bool seed = valid && P.tstamp[g] == 1;
        warp_push(P.ctl, &P.ctl->rcnt[0], P.list0, P.n_tiles, seed, g, P.ordered ? &P.ctl->rkmin[0] : nullptr, key);
    }
}

// Sources: tau = -1 marker (lambda stays 0 there).
template <class T, int BX, int BY, int BZ>
__global__ void k_adj_sources(AdjParams<T> P) {
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
    const int g = (int)(d.tile_base + ((long long)(k / BZ) * d.ty + (j / BY)) * d.tx + (i / BX));
    const int loc = ((k % BZ) * BY + (j % BY)) * BX + (i % BX);
    P.tau_t[(size_t)g * G::V + loc] = T(-1);
}

// Faces (of fb, the faces of node (x, y, z)) across which the node's lambda
// feeds the node beyond: node p enters the row of its neighbour q across a
// face of the transposed system only if p selects q as its upwind neighbour on
// that axis (q the smaller of p's two neighbours there, a tie to the lower
// index, and phi_p > phi_q); otherwise w_{p->q} = 0 and a change of lambda_p
// leaves q's equation as it was, so the tile beyond need not be listed for it.
// phi is fixed during the adjoint, so the test is exact.
template <class T, int BX, int BY, int BZ>
__device__ __forceinline__ int adj_feeds(const T *phi, int x, int y, int z, int fb) {
    using A = AdjGeom<BX, BY, BZ>;
    const T pj = phi[A::pidx(x, y, z)];
    int r = 0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (!(fb >> (2 * ax) & 3)) continue;
        const int ex = ax == 0, ey = ax == 1, ez = ax == 2;
        const T lo = phi[A::pidx(x - ex, y - ey, z - ez)];
        const T hi = phi[A::pidx(x + ex, y + ey, z + ez)];
        if ((fb >> (2 * ax) & 1) && lo <= hi && lo < pj) r |= 1 << (2 * ax);
        if ((fb >> (2 * ax + 1) & 1) && hi < lo && hi < pj) r |= 2 << (2 * ax);
    }
    return r;
}

// One visit of tile g by a group of GT threads (one or two nodes each).
template <class T, int BX, int BY, int BZ>
__device__ __forceinline__ int adj_visit(const AdjParams<T> &P, AdjSmem<T, BX, BY, BZ> &sm, const int (&nb)[6], int g,
                                         int gt, int bid, unsigned &mine, bool &first_changed) {
    using G = TileGeom<BX, BY, BZ>;
    using A = AdjGeom<BX, BY, BZ>;
    using GG = AdjGroupGeom<BX, BY, BZ>;
    constexpr int NPT = GG::NPT;
    const T INF = Num<T>::inf();
    T lam[NPT], rr[NPT], tau[NPT], J[NPT], w[NPT][6];
    int x[NPT], y[NPT], z[NPT];
    // interior
#pragma unroll
    for (int m = 0; m < NPT; ++m) {
        const int q = GG::node(gt, m);
        x[m] = q % BX; y[m] = (q / BX) % BY; z[m] = q / (BX * BY);
        const size_t a = (size_t)g * G::V + q;
        const T ph = __ldcg(P.phi_t + a);
        lam[m] = __ldcg(P.lam_t + a);
        rr[m] = __ldcg(P.r_t + a);
        tau[m] = __ldcg(P.tau_t + a);
        sm.phi[A::pidx(x[m], y[m], z[m])] = ph;
        sm.lam[G::sidx(x[m], y[m], z[m])] = lam[m];
    }
    // halos: phi two nodes deep, lambda one node deep, on the six faces
    constexpr int FX = BY * BZ, FY = BX * BZ, FZ = BX * BY;
    constexpr int HN = 2 * (FX + FY + FZ);
    for (int e = gt; e < 2 * HN; e += GG::GT) {
        const int depth = e / HN;                 // 0: adjacent layer, 1: second layer
        int f, a, b2, r = e % HN;
        if (r < 2 * FX) { f = r / FX; r %= FX; a = r % BY; b2 = r / BY; }
        else if ((r -= 2 * FX) < 2 * FY) { f = 2 + r / FY; r %= FY; a = r % BX; b2 = r / BX; }
        else { r -= 2 * FY; f = 4 + r / FZ; r %= FZ; a = r % BX; b2 = r / BX; }
        int sx, sy, sz, lx, ly, lz;                // staged position, node in the neighbour tile
        const int dd = depth;                      // 0 or 1
        switch (f) {
            case 0: sx = -1 - dd; sy = a; sz = b2; lx = BX - 1 - dd; ly = a; lz = b2; break;
            case 1: sx = BX + dd; sy = a; sz = b2; lx = dd; ly = a; lz = b2; break;
            case 2: sx = a; sy = -1 - dd; sz = b2; lx = a; ly = BY - 1 - dd; lz = b2; break;
            case 3: sx = a; sy = BY + dd; sz = b2; lx = a; ly = dd; lz = b2; break;
            case 4: sx = a; sy = b2; sz = -1 - dd; lx = a; ly = b2; lz = BZ - 1 - dd; break;
            default: sx = a; sy = b2; sz = BZ + dd; lx = a; ly = b2; lz = dd; break;
        }
        const int n = (unsigned)nb[f] < (unsigned)P.n_tiles ? nb[f] : -1;
        // a second layer beyond a one-node-thick tile axis lies two tiles away: not staged (+inf),
        // which only matters for BZ == 1 tiles, whose grids have no z neighbours at all
        const bool thin = (f >= 4 && BZ == 1) || (f >= 2 && f < 4 && BY == 1) || (f < 2 && BX == 1);
        T pv = INF, lv = T(0);
        if (n >= 0 && !(dd == 1 && thin)) {
            const size_t src = (size_t)n * G::V + (lz * BY + ly) * BX + lx;
            pv = __ldcg(P.phi_t + src);
            if (dd == 0) lv = __ldcg(P.lam_t + src);
        }
        sm.phi[A::pidx(sx, sy, sz)] = pv;
        if (dd == 0) sm.lam[G::sidx(sx, sy, sz)] = lv;
    }
    group_sync(bid, GG::GT);
    // J_jj and the weights w_{i->j} of the six neighbours i = j + e (order -x,+x,-y,+y,-z,+z)
#pragma unroll
    for (int m = 0; m < NPT; ++m) {
        const T pj = sm.phi[A::pidx(x[m], y[m], z[m])];
        J[m] = T(0);
#pragma unroll
        for (int k = 0; k < 6; ++k) w[m][k] = T(0);
        if (tau[m] < T(0) || !(pj < INF) || !(tau[m] < INF)) { J[m] = T(0); continue; }
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const int ex = ax == 0, ey = ax == 1, ez = ax == 2;
            const T lo1 = sm.phi[A::pidx(x[m] - ex, y[m] - ey, z[m] - ez)];
            const T hi1 = sm.phi[A::pidx(x[m] + ex, y[m] + ey, z[m] + ez)];
            const T lo2 = sm.phi[A::pidx(x[m] - 2 * ex, y[m] - 2 * ey, z[m] - 2 * ez)];
            const T hi2 = sm.phi[A::pidx(x[m] + 2 * ex, y[m] + 2 * ey, z[m] + 2 * ez)];
            const T mv = vmin(lo1, hi1);
            if (mv < INF && pj > mv) J[m] += T(2) * (pj - mv);
            // neighbour i = j - e selects j iff phi_j < phi_{j-2e} (a tie goes to the lower index j-2e)
            if (lo1 < INF && pj < lo2 && lo1 > pj) w[m][2 * ax] = T(2) * (lo1 - pj);
            // neighbour i = j + e selects j iff phi_j <= phi_{j+2e} (a tie goes to the lower index j)
            if (hi1 < INF && pj <= hi2 && hi1 > pj) w[m][2 * ax + 1] = T(2) * (hi1 - pj);
        }
    }
    // 1 / J_jj once per visit: a sweep multiplies (the FP32 division in every sweep made the
    // whole adjoint 1.26x slower on the 192^3 tomography batch)
    T rJ[NPT];
#pragma unroll
    for (int m = 0; m < NPT; ++m) rJ[m] = J[m] > T(0) ? T(1) / J[m] : T(0);
    // Sweeps on lambda until no change; sources and nodes with J == 0 keep
    // lambda.  A thread relaxes its z segment in descending z: lambda flows
    // toward lower phi, most often up the grid from receivers below the
    // sources (measured on the 192^3 tomography batch: 15 % faster than
    // slots two z planes apart, 3 % faster than a per-visit vote on the
    // direction).
    mine = 0;
    first_changed = false;
    int s = 0;
    for (;;) {
        unsigned ch = 0;
        // a node with J == 0 (a source, an unreachable or impassable node) has rJ = 0 and zero
        // weights, so its update is 0 * (finite sum) = 0 = its lambda: no test per node
        auto relax = [&](int m) {
            const int c = G::sidx(x[m], y[m], z[m]);
            T acc = rr[m];
            acc += w[m][0] * sm.lam[c - 1];
            acc += w[m][1] * sm.lam[c + 1];
            acc += w[m][2] * sm.lam[c - G::SX];
            acc += w[m][3] * sm.lam[c + G::SX];
            // z neighbours inside the thread's own segment come from registers
            const T lzlo = (GG::ZSEG && m > 0) ? lam[m > 0 ? m - 1 : 0] : sm.lam[c - G::SX * G::SY];
            const T lzhi = (GG::ZSEG && m + 1 < NPT) ? lam[m + 1 < NPT ? m + 1 : m] : sm.lam[c + G::SX * G::SY];
            acc += w[m][4] * lzlo;
            acc += w[m][5] * lzhi;
            const T nl = acc * rJ[m];
            if (nl != lam[m]) { lam[m] = nl; sm.lam[c] = nl; ch |= 1u << m; }
        };
#pragma unroll
        for (int m = NPT - 1; m >= 0; --m) relax(m);
        mine |= ch;
        ++s;
        const int any = group_sync_or(bid, GG::GT, ch != 0);
        if (s == 1) first_changed = any != 0;
        if (!any || s >= P.max_sweeps) break;
    }
#pragma unroll
    for (int m = 0; m < NPT; ++m)
        if (mine >> m & 1) {
            dbg_nan(P.ctl, lam[m]);
            __stcg(P.lam_t + (size_t)g * G::V + GG::node(gt, m), lam[m]);
        }
    return s;
}

// 3 resident CTAs per SM in FP32 (measured on the 192^3 tomography batch: 2 -> 3 is
// 1.08x faster, 4 is slower, with spills); 2 in the FP64 validation mode
template <class T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(32 * kWarpsPerCta, (sizeof(T) == 8 ? 2 : 3)) k_adj_persistent(AdjParams<T> P) {
    using G = TileGeom<BX, BY, BZ>;
    using GG = AdjGroupGeom<BX, BY, BZ>;
    extern __shared__ __align__(16) unsigned char adj_smem_raw[];
    AdjSmem<T, BX, BY, BZ> *sms = reinterpret_cast<AdjSmem<T, BX, BY, BZ> *>(adj_smem_raw);
    __shared__ int s_n, s_p, s_visits;
    __shared__ unsigned s_k;
    __shared__ int s_nb[GG::NG][6];
    __shared__ int s_fmask[GG::NG];
    __shared__ GroupQueue gqs[GG::NG];
    const int gi = threadIdx.x / GG::GT, gt = threadIdx.x % GG::GT, bid = 1 + gi;
    AdjSmem<T, BX, BY, BZ> &sm = sms[gi];
    // faces that never get loaded stay +inf / 0 (z of 2D tiles, far corners)
    for (int q = gt; q < AdjGeom<BX, BY, BZ>::PS; q += GG::GT) sm.phi[q] = Num<T>::inf();
    for (int q = gt; q < G::S; q += GG::GT) sm.lam[q] = T(0);
    if (threadIdx.x == 0) s_visits = 0;
    Ctl *ctl = P.ctl;
    unsigned long long target = 0;
    long long tiles = 0, sweeps = 0, deferred = 0;
    const int groups = gridDim.x * GG::NG;
    float width = 1.0f;
    int n_prev = 0;
    int r = 0;
    __syncthreads();
    for (;; ++r) {
        if (threadIdx.x == 0) {
            s_n = ld_volatile(&ctl->rcnt[r % 3]);
            s_k = ld_volatile_u(&ctl->rkmin[r % 3]);
            s_p = r > 0 ? ld_volatile(&ctl->nproc[(r - 1) % 4]) : 0;
        }
        __syncthreads();
        const int n = min(s_n, P.n_tiles);
        if (r > 0) width = adapt_window(width, s_p, n_prev, groups, groups);
        const int chunk = group_chunk(n, r > 0 ? s_p : 0, r > 0 ? n_prev : 0, groups, GG::GT);
        n_prev = n;
        if (n == 0) break;
        if (r >= P.max_iters) { if (threadIdx.x == 0) atomicOr(&ctl->flags, kFlagCap); break; }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctl->rcnt[(r + 2) % 3] = 0;
            ctl->rkmin[(r + 2) % 3] = kKeyInf;
            ctl->rgrab[(r + 2) % 3] = 0;
            ctl->rvcnt[(r + 2) % 3] = 0;
            ctl->rvgrab[(r + 2) % 3] = 0;
            ctl->nproc[(r + 2) % 4] = 0;
        }
        const OrderCtx ord = order_begin(P.ordered, s_k, width);
        const int nslot = (r + 1) % 3;
        const int *in = (r & 1) ? P.list1 : P.list0;
        int *out = (r & 1) ? P.list0 : P.list1;
        const int next_stamp = r + 2;
        // Visit of tile g (its neighbours in s_nb[gi]) and the listing of the neighbour
        // tiles across faces where a changed lambda feeds the node beyond (adj_feeds).
        auto visit = [&](int g) {
            int nb[6];
#pragma unroll
            for (int f = 0; f < 6; ++f) nb[f] = s_nb[gi][f];
            unsigned mine;
            bool changed;
            const int s = adj_visit<T, BX, BY, BZ>(P, sm, nb, g, gt, bid, mine, changed);
            if (gt == 0) { tiles++; sweeps += s; atomicAdd(&s_visits, 1); }
#pragma unroll
            for (int m = 0; m < GG::NPT; ++m)
                if (mine >> m & 1) {
                    const int q = GG::node(gt, m);
                    int fb = G::faces_of(q);
                    if (fb) fb = adj_feeds<T, BX, BY, BZ>(sm.phi, q % BX, (q / BX) % BY, q / (BX * BY), fb);
                    if (fb) atomicOr(&s_fmask[gi], fb);
                }
            group_sync(bid, GG::GT);
            if (gt < 32) {
                const int fm = s_fmask[gi];
                int cand = -1;
                if (gt < 6 && (fm >> gt & 1) && (unsigned)nb[gt] < (unsigned)P.n_tiles) cand = nb[gt];
                if (gt == 6 && changed && s >= P.max_sweeps) cand = g;
                const unsigned kc = (ord.on && cand >= 0) ? __ldg(P.tkey + cand) : kKeyInf;
                const bool want = cand >= 0 && atomicExch(P.tstamp + cand, next_stamp) != next_stamp;
                warp_push(ctl, &ctl->rcnt[nslot], out, P.n_tiles, want, cand, ord.on ? &ctl->rkmin[nslot] : nullptr, kc);
            }
            group_sync(bid, GG::GT);                       // the visit is done with s_nb, s_fmask and sm
        };
        if ((r > 0 ? s_p : n) > groups) {
            // more visits expected than groups: two phases split by a grid barrier (as the
            // forward's group_pass_split): every thread classifies list entries, a kept tile
            // goes to the visit list with its neighbours; then the groups take one visit at a time
            const int lane = threadIdx.x & 31;
            const int nthreads = gridDim.x * blockDim.x;
            int *vcnt = &ctl->rvcnt[r % 3];
            for (int e0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); e0 < n; e0 += nthreads) {
                const int e = e0 + lane;
                bool valid = e < n;
                const int g = valid ? __ldcg(in + e) : -1;
                if (valid && dbg_bad_tile(ctl, g, P.n_tiles)) valid = false;
                int4 r0 = make_int4(0, 0, 0, 0), r1 = r0;
                if (valid) {
                    r0 = __ldcg(reinterpret_cast<const int4 *>(P.tile_rec + 8 * g));
                    r1 = __ldcg(reinterpret_cast<const int4 *>(P.tile_rec + 8 * g + 4));
                }
                const unsigned key = valid && ord.on ? __ldg(P.tkey + g) : kKeyInf;
                const bool defer = valid && ord.on && !order_visit(ord, key);
                bool want = false;
                if (defer) {                               // deferred: listed again, not visited
                    want = atomicExch(P.tstamp + g, next_stamp) != next_stamp;
                    deferred++;
                }
                warp_push(ctl, &ctl->rcnt[nslot], out, P.n_tiles, want, g, ord.on ? &ctl->rkmin[nslot] : nullptr, key);
                push_visit(ctl, vcnt, P.vlist, P.n_tiles, valid && !defer, g, key, r0, r1);
            }
            if (!grid_sync(ctl, target, P.wait_ns)) break;
            const int nv = min(ld_volatile(vcnt), P.n_tiles);
            __shared__ int s_tile[GG::NG];
            for (bool first = true;; first = false) {
                if (gt == 0) {
                    const int idx = first ? blockIdx.x * GG::NG + gi : groups + atomicAdd(&ctl->rvgrab[r % 3], 1);
                    int g = -1;
                    if (idx < nv) {
                        const VisitRec *vr = P.vlist + idx;
                        g = __ldcg(&vr->head).x;
                        if (dbg_bad_tile(ctl, g, P.n_tiles)) g = -1;
                        const int4 a = __ldcg(&vr->r0), b = __ldcg(&vr->r1);
                        s_nb[gi][0] = a.x; s_nb[gi][1] = a.y; s_nb[gi][2] = a.z; s_nb[gi][3] = a.w;
                        s_nb[gi][4] = b.x; s_nb[gi][5] = b.y;
                        s_fmask[gi] = 0;
                    }
                    s_tile[gi] = g;
                }
                group_sync(bid, GG::GT);
                const int g = s_tile[gi];
                if (g < 0) break;                          // group-uniform
                visit(g);
            }
        } else {
            // groups take chunks of the list from a shared counter, classify a chunk
            // with all their threads (deferred entries are listed again on the spot)
            // and visit the kept tiles one by one
            GroupQueue &q = gqs[gi];
            int *grab = &ctl->rgrab[r % 3];
            // the static first chunks cover the list: no grab from the shared counter
            const bool static_only = (long long)gridDim.x * GG::NG * chunk >= n;
            for (bool first = true;; first = false) {
                if (!first && static_only) break;
                if (gt == 0) {
                    q.n = 0;
                    q.base = grab_chunk(grab, first, blockIdx.x * GG::NG + gi, gridDim.x * GG::NG, chunk);
                }
                group_sync(bid, GG::GT);
                const int base = q.base;
                if (base >= n) break;                          // group-uniform
                {
                    const int e = base + gt;
                    bool valid = gt < chunk && e < n;
                    const int g = valid ? __ldcg(in + e) : -1;
                    if (valid && dbg_bad_tile(ctl, g, P.n_tiles)) valid = false;
                    const unsigned key = valid && ord.on ? __ldg(P.tkey + g) : kKeyInf;
                    const bool defer = valid && ord.on && !order_visit(ord, key);
                    bool want = false;
                    if (defer) {                               // deferred: listed again, not visited
                        want = atomicExch(P.tstamp + g, next_stamp) != next_stamp;
                        deferred++;
                    }
                    warp_push(ctl, &ctl->rcnt[nslot], out, P.n_tiles, want, g, ord.on ? &ctl->rkmin[nslot] : nullptr, key);
                    if (valid && !defer) q.tile[atomicAdd(&q.n, 1)] = g;
                }
                group_sync(bid, GG::GT);
                const int qn = q.n;
                for (int qi = 0; qi < qn; ++qi) {
                    const int g = q.tile[qi];
                    if (gt == 0) {
#pragma unroll
                        for (int f = 0; f < 6; ++f) s_nb[gi][f] = __ldcg(P.tile_rec + 8 * g + f);
                        s_fmask[gi] = 0;
                    }
                    group_sync(bid, GG::GT);
                    visit(g);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_visits) { atomicAdd(&ctl->nproc[r % 4], s_visits); s_visits = 0; }
        if (!grid_sync(ctl, target, P.wait_ns)) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->iters_remedy = r;
    // visits and sweeps are counted by thread 0 of each group, deferrals by the classifying threads
    if (tiles) atomicAdd((unsigned long long *)&ctl->tiles_remedy, (unsigned long long)tiles);
    if (sweeps) atomicAdd((unsigned long long *)&ctl->sweeps, (unsigned long long)sweeps);
    if (deferred) atomicAdd((unsigned long long *)&ctl->tiles_deferred, (unsigned long long)deferred);
}

// g_out[block][node] += sum over the instances b writing that gradient block,
// in instance order, of 2 h tau_b lambda_b, at non-source nodes with finite
// phi and tau (blocks are equal or disjoint, so one thread owns each node: the
// sum has a fixed order and no atomics).  A CTA takes kSpan consecutive tiles
// of the blocks (of their first instances) at a time; every thread loads its
// nodes of each instance at once.
template <class T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(kSpanThreads) k_adj_output(AdjParams<T> P) {
    using G = TileGeom<BX, BY, BZ>;
    constexpr int PER = kSpan * G::V / kSpanThreads;
    __shared__ TileSpan<BX, BY, BZ> sp;
    for (long long a0 = (long long)blockIdx.x * kSpan; a0 < P.n_acc_tiles; a0 += (long long)gridDim.x * kSpan) {
        if (threadIdx.x < kSpan) sp.fill(P.desc, P.B, P.n_acc_tiles, a0, threadIdx.x, true);
        __syncthreads();
        // instance of each tile's chain being added (-1: done); every thread walks the chains itself
        int bt[kSpan];
#pragma unroll
        for (int t = 0; t < kSpan; ++t) bt[t] = a0 + t < P.n_acc_tiles ? sp.inst[t] : -1;
        T sum[PER];
        bool any[PER];
#pragma unroll
        for (int m = 0; m < PER; ++m) { sum[m] = T(0); any[m] = false; }
        for (;;) {
            bool live = false;
#pragma unroll
            for (int t = 0; t < kSpan; ++t) live |= bt[t] >= 0;
            if (!live) break;                                       // uniform: every thread walks the same chains
            T lam[PER], h2[PER];
            long long e[PER];
#pragma unroll
            for (int m = 0; m < PER; ++m) {
                const int r = threadIdx.x + m * kSpanThreads, t = r / G::V, q = r % G::V;
                int b = bt[0];
#pragma unroll
                for (int u = 1; u < kSpan; ++u) b = t == u ? bt[u] : b;
                lam[m] = T(0); h2[m] = T(0); e[m] = -1;
                if (b < 0) continue;
                e[m] = (P.desc[b].tile_base + sp.l[t]) * G::V + q;
                lam[m] = __ldcs(P.lam_t + e[m]);
                h2[m] = T(2) * T(P.desc[b].h);
            }
            // lambda != 0 only at non-source nodes with finite phi and tau (the visits keep
            // lambda = 0 elsewhere): tau is read only there
#pragma unroll
            for (int m = 0; m < PER; ++m) {
                if (lam[m] == T(0)) continue;
                const T tau = __ldcs(P.tau_t + e[m]);
                if (tau < T(0) || !(tau < Num<T>::inf())) continue;
                sum[m] += h2[m] * tau * lam[m];
                any[m] = true;
            }
#pragma unroll
            for (int t = 0; t < kSpan; ++t)
                if (bt[t] >= 0) bt[t] = P.desc[bt[t]].acc_next;
        }
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int r = threadIdx.x + m * kSpanThreads, t = r / G::V, q = r % G::V;
            const int x = q % BX, y = (q / BX) % BY, z = q / (BX * BY);
            if (!any[m] || !sp.inside(t, x, y, z)) continue;
            T *o = P.g_out + P.desc[sp.inst[t]].aux_off + sp.at(t, x, y, z);
            *o += sum[m];
        }
        __syncthreads();                                            // the span is refilled next
    }
}

}  // namespace eik
