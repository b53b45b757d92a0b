// eik_api.cu -- the C ABI of libeikonal.so (declared in include/eikonal.h):
// argument checks, workspace layout, template dispatch over precision and
// tile shape, and the two loop schedules (persistent cooperative launch, or
// one launch per iteration with a host-read list size).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/eikonal.h"
#include "eik_common.cuh"
#include "eik_kernels.cuh"
#include "eik_async.cuh"
#include "eik_adjoint.cuh"
#include "eik_backtrace.cuh"

using namespace eik;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(EIK_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define EIK_CUDA(call, what)                         \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

struct TileShape {
    int bx, by, bz;
};

TileShape tile_shape(int tile) {
    switch (tile) {
        case EIK_TILE_4x4x4: return {4, 4, 4};
        case EIK_TILE_8x8x4: return {8, 8, 4};
        case EIK_TILE_16x16x1: return {16, 16, 1};
        case EIK_TILE_8x4x4: return {8, 4, 4};
        case EIK_TILE_8x8x1: return {8, 8, 1};
        default: return {8, 8, 8};
    }
}

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Opts {
    int tile, schedule, precision, skip_remedy, converge, method;
    long long max_iters;
    unsigned long long wait_ns;   // bound on every device wait (kWaitLimitNs unless the call sets one)
    float order;           // <= 0: unordered lists (every listed tile visited each iteration)
    bool order_update;     // the Step-2 lists are bucketed too
};

constexpr float kDefaultOrder = 4.0f;          // bucket width (tile-crossing times) of the default schedule
// the adjoint's default window (its keys are static).  Measured on B300 on the 16-shot 192^3
// tomography with the adjoint's listing test: width 1 / 2 / 3 / 4 / 8 -> 6.08 / 5.71 / 5.83 /
// 5.98 / 6.78 ms (the gradient is the same bit for bit)
constexpr float kDefaultAdjointOrder = 2.0f;

bool read_opts(const eik_options *o, int64_t B, const eik_grid *grids, Opts &out) {
    out.tile = o ? o->tile : EIK_TILE_AUTO;
    out.schedule = o ? o->schedule : EIK_SCHED_AUTO;
    out.precision = o ? o->precision : EIK_FP32;
    out.skip_remedy = o ? o->skip_remedy : 0;
    out.max_iters = o ? o->max_iters : 0;
    const float ord = o ? o->order : 0.0f;
    if (!(ord == ord)) return false;                       // NaN
    out.order = ord == 0.0f ? kDefaultOrder : (ord < 0.0f ? 0.0f : ord);
    out.converge = o ? o->converge : EIK_CONVERGE_AUTO;
    if (out.converge < 0 || out.converge > EIK_CONVERGE_SWEEP) return false;
    if (out.converge == EIK_CONVERGE_AUTO) out.converge = EIK_CONVERGE_CONFIRM;
    out.method = o ? o->method : EIK_METHOD_IFIM;
    if (out.method != EIK_METHOD_IFIM && out.method != EIK_METHOD_FIM) return false;
    if (out.method == EIK_METHOD_FIM) {
        out.converge = EIK_CONVERGE_SWEEP;                  // a visit relaxes to the tile's local fixed point
        out.skip_remedy = 0;
    }
    const long long wl = o ? (long long)o->wait_limit_us : 0;
    if (wl < 0) return false;
    out.wait_ns = wl > 0 ? (unsigned long long)wl * 1000ull : kWaitLimitNs;
    if (out.precision != EIK_FP32 && out.precision != EIK_FP64) return false;
    if (out.schedule < 0 || out.schedule > EIK_SCHED_ASYNC) return false;
    if (out.tile < 0 || out.tile > EIK_TILE_8x8x1) return false;
    bool all2d = true;
    for (int64_t b = 0; b < B; ++b) all2d = all2d && grids[b].nz == 1;
    // Default list order: the Step-3 (and FIM) lists bucketed with width kDefaultOrder; the
    // Step-2 lists bucketed too on 2D grids, unordered on 3D grids (every Active tile visited
    // in every iteration, as Algorithm 2 is printed).  Measured on B300: unordered Step-2
    // lists take the 512^3 maze from 38.6 to 24.3 ms and the 256^3 oscillating speed from
    // 6.7 to 6.1 ms, while Example 5 at 4000^2 goes from 11.2 to 16.0 ms.  An explicit
    // order > 0 buckets both loops with that width, < 0 neither.
    out.order_update = ord > 0.0f || (ord == 0.0f && all2d);
    const float rord = o ? o->remedy_order : 0.0f;
    if (!(rord == rord)) return false;                     // NaN
    if (!out.order_update && rord != 0.0f) out.order = rord > 0.0f ? rord : 0.0f;
    if (out.tile == EIK_TILE_AUTO) out.tile = all2d ? EIK_TILE_16x16x1 : EIK_TILE_8x8x8;
    if ((out.tile == EIK_TILE_16x16x1 || out.tile == EIK_TILE_8x8x1) && !all2d) return false;
    if (out.max_iters < 0) return false;
    return true;
}

// workspace regions (byte offsets), all 256-byte aligned
struct Layout {
    size_t ctl, desc, tile_fstat, inst_scale, scale_part, scale_done, tile_inst, tile_nb, tstate, tstamp, tkey, list0,
        list1, vlist, phi_t, tau_t;
    size_t q_data, q_seq, q_state, total;
    long long n_tiles;
    unsigned long long q_slots;
    std::vector<InstDesc> desc_host;
    double cy = 1.0, cz = 1.0;   // axis weights (dx/dy)^2, (dx/dz)^2 shared by the call's grids
    bool aniso = false;
};

// spacing along y and z of a grid (0 = h)
inline double spacing_y(const eik_grid &g) { return g.hy != 0.0 ? g.hy : g.h; }
inline double spacing_z(const eik_grid &g) { return g.hz != 0.0 ? g.hz : g.h; }
inline bool spacing_ok(double v) { return v == 0.0 || (v > 0.0 && v < 1e300); }

bool make_layout(int64_t B, const eik_grid *grids, const Opts &o, Layout &L, std::string *why) {
    const TileShape ts = tile_shape(o.tile);
    const size_t esz = o.precision == EIK_FP64 ? 8 : 4;
    const long long V = (long long)ts.bx * ts.by * ts.bz;
    L.desc_host.resize((size_t)B);
    L.cy = L.cz = 1.0;
    bool have_cy = false, have_cz = false;
    long long tiles = 0;
    for (int64_t b = 0; b < B; ++b) {
        const eik_grid &g = grids[b];
        if (g.nx < 1 || g.ny < 1 || g.nz < 1 || g.nx > (1ll << 30) || g.ny > (1ll << 30) || g.nz > (1ll << 30)) {
            if (why) *why = "grid " + std::to_string(b) + ": dims must be in [1, 2^30]";
            return false;
        }
        if (!(g.h > 0.0) || !(g.h < 1e300)) {
            if (why) *why = "grid " + std::to_string(b) + ": h must be finite and > 0";
            return false;
        }
        if (!spacing_ok(g.hy) || !spacing_ok(g.hz)) {
            if (why) *why = "grid " + std::to_string(b) + ": hy, hz must be 0 or finite and > 0";
            return false;
        }
        {
            // axis weights, compared over the grids that have that axis
            const double ry = g.h / spacing_y(g), rz = g.h / spacing_z(g);
            const double cyb = ry * ry, czb = rz * rz;
            if ((g.ny > 1 && have_cy && cyb != L.cy) || (g.nz > 1 && have_cz && czb != L.cz)) {
                if (why) *why = "grid " + std::to_string(b) + ": all grids of one call must have the same hy/h and hz/h";
                return false;
            }
            if (g.ny > 1 && !have_cy) { L.cy = cyb; have_cy = true; }
            if (g.nz > 1 && !have_cz) { L.cz = czb; have_cz = true; }
        }
        InstDesc &d = L.desc_host[(size_t)b];
        std::memset(&d, 0, sizeof(d));
        d.nx = (int)g.nx; d.ny = (int)g.ny; d.nz = (int)g.nz;
        d.tx = (int)((g.nx + ts.bx - 1) / ts.bx);
        d.ty = (int)((g.ny + ts.by - 1) / ts.by);
        d.tz = (int)((g.nz + ts.bz - 1) / ts.bz);
        d.tile_base = tiles;
        d.acc_base = tiles;
        d.acc_next = -1;
        d.h = g.h;
        tiles += (long long)d.tx * d.ty * d.tz;
        if (tiles >= (1ll << 31) - 1) {
            if (why) *why = "too many tiles (more than 2^31 - 2)";
            return false;
        }
    }
    L.aniso = L.cy != 1.0 || L.cz != 1.0;
    L.n_tiles = tiles;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o2 = off; off = align_up(off + bytes, 256); return o2; };
    L.ctl = take(sizeof(Ctl));
    L.desc = take(sizeof(InstDesc) * (size_t)B);
    L.inst_scale = take(sizeof(float) * (size_t)B);
    L.scale_part = take(sizeof(ScalePart) * (size_t)scale_chunks(B) * (size_t)B);
    L.scale_done = take(sizeof(int) * (size_t)B);
    L.tile_inst = take(4 * (size_t)tiles);
    L.tile_nb = take(4 * 8 * (size_t)tiles);
    L.tile_fstat = take(8 * (size_t)tiles);
    L.tstate = take(4 * (size_t)tiles);
    L.tstamp = take(4 * (size_t)tiles);
    L.tkey = take(2 * 4 * (size_t)tiles);
    L.list0 = take(4 * (size_t)tiles);
    L.list1 = take(4 * (size_t)tiles);
    L.vlist = take(sizeof(VisitRec) * (size_t)tiles);
    L.phi_t = take(esz * (size_t)(tiles * V));
    L.tau_t = take(esz * (size_t)(tiles * V));
    // work queue of the asynchronous schedule: 2^k slots > tiles + any number of warps
    // (only when that schedule may run: explicitly requested, or chosen by auto)
    unsigned long long q = 1;
    const bool need_q = o.schedule == EIK_SCHED_ASYNC || o.schedule == EIK_SCHED_AUTO;
    if (need_q)
        while (q < 2ull * (unsigned long long)tiles + 65536ull) q <<= 1;
    L.q_slots = need_q ? q : 0;
    L.q_data = take(4 * (size_t)L.q_slots);
    L.q_seq = take(8 * (size_t)L.q_slots);
    L.q_state = take(need_q ? 4 * (size_t)tiles : 0);
    L.total = off;
    return true;
}

long long auto_max_iters(const Layout &L) {
    long long m = 0;
    for (const InstDesc &d : L.desc_host) {
        const long long s = (long long)d.tx + d.ty + d.tz;
        if (s > m) m = s;
    }
    return 64 * m + 4096;
}

struct DevInfo {
    int dev = -1, sms = 0, coop = 0;
};

int device_info(DevInfo &di) {
    EIK_CUDA(cudaGetDevice(&di.dev), "cudaGetDevice");
    EIK_CUDA(cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, di.dev), "cudaDeviceGetAttribute");
    EIK_CUDA(cudaDeviceGetAttribute(&di.coop, cudaDevAttrCooperativeLaunch, di.dev), "cudaDeviceGetAttribute");
    return EIK_OK;
}

int upload_desc(InstDesc *ddesc, const std::vector<InstDesc> &h, cudaStream_t st) {
    const int B = (int)h.size();
    for (int first = 0; first < B; first += kMaxInstPerLaunch) {
        DescChunk c;
        std::memset(&c, 0, sizeof(c));
        c.first = first;
        c.count = std::min(kMaxInstPerLaunch, B - first);
        for (int q = 0; q < c.count; ++q) c.d[q] = h[(size_t)(first + q)];
        k_write_desc<<<1, kMaxInstPerLaunch, 0, st>>>(ddesc, c);
        EIK_CUDA(cudaGetLastError(), "k_write_desc launch");
    }
    return EIK_OK;
}

// CUDA events bracketing the phases of one call (created only when stats are requested)
struct PhaseEvents {
    cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
    bool on = false;
    int create() {
        for (auto &x : e) EIK_CUDA(cudaEventCreate(&x), "cudaEventCreate");
        on = true;
        return EIK_OK;
    }
    void record(int q, cudaStream_t st) {
        if (on) (void)cudaEventRecord(e[q], st);
    }
    ~PhaseEvents() {
        for (auto &x : e)
            if (x) (void)cudaEventDestroy(x);
    }
};

int finish_stats(Ctl *dctl, cudaStream_t st, eik_stats *stats, PhaseEvents *pe) {
    Ctl h;
    EIK_CUDA(cudaMemcpyAsync(&h, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st), "stats copy");
    EIK_CUDA(cudaStreamSynchronize(st), "stream synchronize");
    if (pe && pe->on) {
        float a = 0.f, b = 0.f;
        EIK_CUDA(cudaEventElapsedTime(&a, pe->e[0], pe->e[3]), "cudaEventElapsedTime");
        EIK_CUDA(cudaEventElapsedTime(&b, pe->e[1], pe->e[2]), "cudaEventElapsedTime");
        stats->ms_total = a;
        stats->ms_loop = b;
    }
    stats->iters_update = h.iters_update;
    stats->iters_remedy = h.iters_remedy;
    stats->tiles_update = h.tiles_update;
    stats->tiles_flagged = h.tiles_flagged;
    stats->tiles_remedy = h.tiles_remedy;
    stats->sweeps = h.sweeps;
    stats->tiles_deferred = h.tiles_deferred;
    stats->device_flags = h.flags;
    int code = EIK_OK;
    if (h.flags & kFlagTimeout) code = fail(EIK_ERR_DEVICE, "a device-side wait timed out");
    else if (h.flags & kFlagDebugIndex) code = fail(EIK_ERR_DEVICE, "debug check: a tile id out of range");
    else if (h.flags & kFlagDebugNaN) code = fail(EIK_ERR_DEVICE, "debug check: NaN written to phi or lambda");
    else if (h.flags & kFlagOverflow) code = fail(EIK_ERR_DEVICE, "internal list overflow");
    else if (h.flags & kFlagBadSource) code = fail(EIK_ERR_ARG, "a source index lies outside its grid");
    else if (h.flags & kFlagCap) code = fail(EIK_ERR_NOCONVERGE, "iteration cap reached");
    stats->status = code;
    return code;
}

template <class T, int BX, int BY, int BZ>
int run_forward(const Layout &L, const Opts &o, char *ws, const void *F, const int64_t *src_idx,
                const void *src_val, int64_t n_src, void *phi, cudaStream_t st, eik_stats *stats) {
    FwdParams<T> P;
    P.desc = reinterpret_cast<const InstDesc *>(ws + L.desc);
    P.B = (int)L.desc_host.size();
    P.n_tiles = (int)L.n_tiles;
    P.tile_inst = reinterpret_cast<int *>(ws + L.tile_inst);
    P.tile_nb = reinterpret_cast<int *>(ws + L.tile_nb);
    P.tstate = reinterpret_cast<int *>(ws + L.tstate);
    P.tstamp = reinterpret_cast<int *>(ws + L.tstamp);
    P.tkey = reinterpret_cast<unsigned *>(ws + L.tkey);
    P.inst_scale = reinterpret_cast<float *>(ws + L.inst_scale);
    P.scale_part = reinterpret_cast<ScalePart *>(ws + L.scale_part);
    P.scale_done = reinterpret_cast<int *>(ws + L.scale_done);
    P.tile_fstat = reinterpret_cast<float *>(ws + L.tile_fstat);
    P.ordered = o.order > 0.0f ? 1 : 0;
    P.ordered_update = o.order_update ? 1 : 0;
    P.order = o.order;
    P.list0 = reinterpret_cast<int *>(ws + L.list0);
    P.list1 = reinterpret_cast<int *>(ws + L.list1);
    P.vlist = reinterpret_cast<VisitRec *>(ws + L.vlist);
    P.phi_t = reinterpret_cast<T *>(ws + L.phi_t);
    P.tau_t = reinterpret_cast<T *>(ws + L.tau_t);
    P.ctl = reinterpret_cast<Ctl *>(ws + L.ctl);
    P.max_iters = o.max_iters > 0 ? o.max_iters : auto_max_iters(L);
    P.skip_remedy = o.skip_remedy;
    P.fim = o.method == EIK_METHOD_FIM ? 1 : 0;
    P.mt.cy = (T)L.cy;
    P.mt.cz = (T)L.cz;
    P.mt.aniso = L.aniso ? 1 : 0;
    P.mt.r_xy = (T)(1.0 / (1.0 + L.cy));
    P.mt.r_xz = (T)(1.0 / (1.0 + L.cz));
    P.mt.r_yz = (T)(1.0 / (L.cy + L.cz));
    P.mt.r_xyz = (T)(1.0 / (1.0 + L.cy + L.cz));
    P.one_visit = o.converge == EIK_CONVERGE_SWEEP ? 1 : 0;
    P.max_sweeps = 4 * (BX + BY + BZ) + 8;
    P.F = static_cast<const T *>(F);
    P.src_idx = reinterpret_cast<const long long *>(src_idx);
    P.src_val = static_cast<const T *>(src_val);
    P.n_src = n_src;
    P.phi_out = static_cast<T *>(phi);
    P.wait_ns = o.wait_ns;
    static_assert(sizeof(Ctl) / sizeof(int) <= kSpanThreads, "control block zeroing by the threads of one CTA");

    PhaseEvents pe;
    int rc = EIK_OK;
    if (stats && (rc = pe.create())) return rc;
    pe.record(0, st);
    rc = upload_desc(const_cast<InstDesc *>(P.desc), L.desc_host, st);
    if (rc) return rc;
    {
        DevInfo dinit;
        rc = device_info(dinit);
        if (rc) return rc;
        const long long ctas = std::min<long long>((L.n_tiles + kSpan - 1) / kSpan, 16ll * dinit.sms);
        k_init<T, BX, BY, BZ><<<(unsigned)std::max<long long>(ctas, 1), kSpanThreads, 0, st>>>(P);
        EIK_CUDA(cudaGetLastError(), "k_init launch");
    }
    if (P.ordered) {
        const int chunks = scale_chunks(P.B);
        k_scale<BX, BY, BZ><<<(unsigned)((long long)chunks * P.B), kScaleThreads, 0, st>>>(
            P.desc, reinterpret_cast<const float2 *>(P.tile_fstat), P.inst_scale, P.B, chunks, P.order, P.scale_part,
            P.scale_done);
        EIK_CUDA(cudaGetLastError(), "k_scale launch");
        k_tile_scale<<<(unsigned)std::min<long long>((L.n_tiles + 255) / 256, 4096), 256, 0, st>>>(P.tile_nb, P.inst_scale,
                                                                                               (int)L.n_tiles);
        EIK_CUDA(cudaGetLastError(), "k_tile_scale launch");
    }
    if (n_src > 0) {
        k_sources<T, BX, BY, BZ><<<(unsigned)((n_src + 255) / 256), 256, 0, st>>>(P);
        EIK_CUDA(cudaGetLastError(), "k_sources launch");
    }

    DevInfo di;
    rc = device_info(di);
    if (rc) return rc;
    constexpr int CTA = 32 * kWarpsPerCta;
    // the latency-only persistent kernel for FP32 8x8x8 tiles, the mixed one otherwise
    const void *kpers = (const void *)k_persistent<T, BX, BY, BZ, kPersistMixed>;
    if constexpr (sizeof(T) == 4 && BX * BY * BZ == 512) kpers = (const void *)k_persistent<T, BX, BY, BZ, kPersistLatency>;
    int per_sm = 0, per_sm_pers = 0;
    EIK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent<T, BX, BY, BZ, kPersistMixed>, CTA, 0),
             "occupancy query");
    EIK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_pers, kpers, CTA, 0), "occupancy query");
    int sched = o.schedule;
    if (sched == EIK_SCHED_AUTO) sched = (di.coop && per_sm_pers > 0) ? EIK_SCHED_PERSISTENT : EIK_SCHED_HOSTLOOP;

    bool done = false;
    pe.record(1, st);
    if (sched == EIK_SCHED_ASYNC) {
        AsyncQ Q;
        Q.data = reinterpret_cast<int *>(ws + L.q_data);
        Q.seq = reinterpret_cast<unsigned long long *>(ws + L.q_seq);
        Q.qstate = reinterpret_cast<int *>(ws + L.q_state);
        Q.mask = L.q_slots - 1;
        Q.visit_cap = P.max_iters * (long long)L.n_tiles;
        Q.wait_ns = o.wait_ns;
        Q.n_tiles = (int)L.n_tiles;
        int per_sm_a = 0;
        EIK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_a, k_async<T, BX, BY, BZ>, CTA, 0),
                 "occupancy query");
        if (!di.coop || per_sm_a < 1) return fail(EIK_ERR_CUDA, "the asynchronous schedule needs a cooperative launch");
        k_queue_init<<<std::min<unsigned long long>((L.q_slots + 255) / 256, 4096), 256, 0, st>>>(Q, (int)L.n_tiles);
        EIK_CUDA(cudaGetLastError(), "k_queue_init launch");
        k_queue_seed<<<std::max(1, std::min((int)((L.n_tiles + 255) / 256), 1024)), 256, 0, st>>>(
            Q, P.ctl, P.fim ? &P.ctl->rcnt[0] : &P.ctl->cnt[0], P.list0);
        EIK_CUDA(cudaGetLastError(), "k_queue_seed launch");
        const int grid = per_sm_a * di.sms;
        void *args[] = {&P, &Q};
        EIK_CUDA(cudaLaunchCooperativeKernel((const void *)k_async<T, BX, BY, BZ>, dim3(grid), dim3(CTA), args, 0, st),
                 "cooperative launch");
        done = true;
    }
    if (!done && sched == EIK_SCHED_PERSISTENT) {
        int grid = per_sm_pers * di.sms;
        const int need = (int)((L.n_tiles + kWarpsPerCta - 1) / kWarpsPerCta);
        if (grid > need) grid = need;
        if (grid < 1) grid = 1;
        void *args[] = {&P};
        cudaError_t e = cudaLaunchCooperativeKernel(kpers, dim3(grid), dim3(CTA), args, 0, st);
        if (e == cudaSuccess) {
            done = true;
        } else if (o.schedule == EIK_SCHED_PERSISTENT) {
            return cuda_fail(e, "cooperative launch");
        } else {
            (void)cudaGetLastError();   // clear, then fall back to the host loop
        }
    }
    if (!done) {
        // host loop: one launch per iteration, the list size is read back each time
        const int grid_cap = std::max(1, per_sm * di.sms);
        Ctl *dctl = P.ctl;
        int n = 0, prev_n = 0;
        EIK_CUDA(cudaMemcpyAsync(&n, P.fim ? &dctl->rcnt[0] : &dctl->cnt[0], sizeof(int), cudaMemcpyDeviceToHost, st),
                 "count copy");
        EIK_CUDA(cudaStreamSynchronize(st), "stream synchronize");
        long long it = 0, r = 0;
        bool capped = false;
        while (n > 0 && !P.fim) {
            if (it >= P.max_iters) { capped = true; break; }
            k_update_iter<T, BX, BY, BZ><<<std::min((n + kWarpsPerCta - 1) / kWarpsPerCta, grid_cap), CTA, 0, st>>>(
                P, (int)it, prev_n);
            prev_n = n;
            EIK_CUDA(cudaGetLastError(), "k_update_iter launch");
            ++it;
            EIK_CUDA(cudaMemcpyAsync(&n, &dctl->cnt[it % 3], sizeof(int), cudaMemcpyDeviceToHost, st), "count copy");
            EIK_CUDA(cudaStreamSynchronize(st), "stream synchronize");
        }
        if (!capped && (P.fim || !P.skip_remedy)) {
            if (!P.fim) {
                k_detect<T, BX, BY, BZ><<<std::min((int)((L.n_tiles + kWarpsPerCta - 1) / kWarpsPerCta), grid_cap), CTA,
                                          0, st>>>(P);
                EIK_CUDA(cudaGetLastError(), "k_detect launch");
                EIK_CUDA(cudaMemcpyAsync(&n, &dctl->rcnt[0], sizeof(int), cudaMemcpyDeviceToHost, st), "count copy");
                const int zeros[4] = {0, 0, 0, 0};
                EIK_CUDA(cudaMemcpyAsync(&dctl->nproc[0], zeros, sizeof(zeros), cudaMemcpyHostToDevice, st),
                         "nproc reset");
                EIK_CUDA(cudaStreamSynchronize(st), "stream synchronize");
            }
            // Step 3b, or the one loop of the FIM (entered with the source tiles listed)
            prev_n = 0;
            while (n > 0) {
                if (r >= P.max_iters) { capped = true; break; }
                k_remedy_iter<T, BX, BY, BZ><<<std::min((n + kWarpsPerCta - 1) / kWarpsPerCta, grid_cap), CTA, 0, st>>>(
                    P, (int)r, prev_n);
                prev_n = n;
                EIK_CUDA(cudaGetLastError(), "k_remedy_iter launch");
                ++r;
                EIK_CUDA(cudaMemcpyAsync(&n, &dctl->rcnt[r % 3], sizeof(int), cudaMemcpyDeviceToHost, st),
                         "count copy");
                EIK_CUDA(cudaStreamSynchronize(st), "stream synchronize");
            }
        }
        long long iters[2] = {it, r};
        EIK_CUDA(cudaMemcpyAsync(&dctl->iters_update, iters, sizeof(iters), cudaMemcpyHostToDevice, st),
                 "iters copy");
        if (capped) {
            int f = kFlagCap;
            int cur = 0;
            EIK_CUDA(cudaMemcpyAsync(&cur, &dctl->flags, sizeof(int), cudaMemcpyDeviceToHost, st), "flags copy");
            EIK_CUDA(cudaStreamSynchronize(st), "stream synchronize");
            f |= cur;
            EIK_CUDA(cudaMemcpyAsync(&dctl->flags, &f, sizeof(int), cudaMemcpyHostToDevice, st), "flags copy");
        }
        EIK_CUDA(cudaStreamSynchronize(st), "stream synchronize");
    }
    pe.record(2, st);
    {
        const long long ctas = std::min<long long>((L.n_tiles + kSpan - 1) / kSpan, 16ll * di.sms);
        k_unpack<T, BX, BY, BZ><<<(unsigned)std::max<long long>(ctas, 1), kSpanThreads, 0, st>>>(P);
    }
    EIK_CUDA(cudaGetLastError(), "k_unpack launch");
    pe.record(3, st);
    if (stats) return finish_stats(P.ctl, st, stats, &pe);
    return EIK_OK;
}

template <class T>
int dispatch_tile(const Layout &L, const Opts &o, char *ws, const void *F, const int64_t *si, const void *sv,
                  int64_t ns, void *phi, cudaStream_t st, eik_stats *stats) {
    switch (o.tile) {
        case EIK_TILE_4x4x4: return run_forward<T, 4, 4, 4>(L, o, ws, F, si, sv, ns, phi, st, stats);
        case EIK_TILE_8x8x4: return run_forward<T, 8, 8, 4>(L, o, ws, F, si, sv, ns, phi, st, stats);
        case EIK_TILE_16x16x1: return run_forward<T, 16, 16, 1>(L, o, ws, F, si, sv, ns, phi, st, stats);
        case EIK_TILE_8x4x4: return run_forward<T, 8, 4, 4>(L, o, ws, F, si, sv, ns, phi, st, stats);
        case EIK_TILE_8x8x1: return run_forward<T, 8, 8, 1>(L, o, ws, F, si, sv, ns, phi, st, stats);
        default: return run_forward<T, 8, 8, 8>(L, o, ws, F, si, sv, ns, phi, st, stats);
    }
}

int solve_impl(int64_t B, const eik_grid *grids, const void *F, const int64_t *F_offsets, const int64_t *src_idx,
               const void *src_val, const int64_t *src_offsets, void *phi, const int64_t *phi_offsets, void *ws,
               size_t ws_bytes, void *stream, const eik_options *opt, eik_stats *stats) {
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (B < 1) return fail(EIK_ERR_ARG, "batch size must be >= 1");
    if (B > (1ll << 24)) return fail(EIK_ERR_ARG, "batch size too large");
    if (!grids) return fail(EIK_ERR_ARG, "grids is NULL");
    Opts o;
    if (!read_opts(opt, B, grids, o)) return fail(EIK_ERR_ARG, "invalid options");
    Layout L;
    std::string why;
    if (!make_layout(B, grids, o, L, &why)) return fail(EIK_ERR_ARG, "%s", why.c_str());
    if (!ws) return fail(EIK_ERR_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(EIK_ERR_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < L.total)
        return fail(EIK_ERR_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
    if (!F || !phi) return fail(EIK_ERR_ARG, "F and phi must be non-NULL");
    if (src_offsets[0] != 0) return fail(EIK_ERR_ARG, "src_offsets[0] must be 0");
    for (int64_t b = 0; b < B; ++b) {
        if (src_offsets[b + 1] < src_offsets[b]) return fail(EIK_ERR_ARG, "src_offsets must be non-decreasing");
        if (F_offsets[b] < 0 || phi_offsets[b] < 0) return fail(EIK_ERR_ARG, "offsets must be >= 0");
        InstDesc &d = L.desc_host[(size_t)b];
        d.in_off = F_offsets[b];
        d.out_off = phi_offsets[b];
        d.src_begin = src_offsets[b];
        d.src_end = src_offsets[b + 1];
    }
    const int64_t n_src = src_offsets[B];
    if (n_src > 0 && (!src_idx || !src_val)) return fail(EIK_ERR_ARG, "source arrays must be non-NULL");
    if (n_src >= (1ll << 40)) return fail(EIK_ERR_ARG, "too many sources");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(ws);
    if (o.precision == EIK_FP64)
        return dispatch_tile<double>(L, o, w, F, src_idx, src_val, n_src, phi, st, stats);
    return dispatch_tile<float>(L, o, w, F, src_idx, src_val, n_src, phi, st, stats);
}

// ---------------------------------------------------------------- adjoint
struct AdjLayout {
    size_t ctl, desc, inst_scale, tile_rec, tstamp, tkey, list0, list1, vlist, phi_t, tau_t, lam_t, r_t, total;
    long long n_tiles;
    long long n_acc_tiles;        // tiles of the distinct gradient blocks
    std::vector<InstDesc> desc_host;
};

bool make_adj_layout(int64_t B, const eik_grid *grids, const Opts &o, AdjLayout &L, std::string *why) {
    Layout fl;   // reuse the forward's dims/tile checks and descriptors
    if (!make_layout(B, grids, o, fl, why)) return false;
    if (fl.aniso) {
        if (why) *why = "the adjoint takes equal spacings (hy = hz = h)";
        return false;
    }
    const TileShape ts = tile_shape(o.tile);
    const size_t esz = o.precision == EIK_FP64 ? 8 : 4;
    const long long V = (long long)ts.bx * ts.by * ts.bz;
    L.desc_host = fl.desc_host;
    L.n_tiles = fl.n_tiles;
    L.n_acc_tiles = fl.n_tiles;   // every instance its own block until chain_gradient_blocks
    const long long tiles = fl.n_tiles;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o2 = off; off = align_up(off + bytes, 256); return o2; };
    L.ctl = take(sizeof(Ctl));
    L.desc = take(sizeof(InstDesc) * (size_t)B);
    L.inst_scale = take(sizeof(float) * (size_t)B);
    L.tile_rec = take(4 * 8 * (size_t)tiles);
    L.tstamp = take(4 * (size_t)tiles);
    L.tkey = take(4 * (size_t)tiles);
    L.list0 = take(4 * (size_t)tiles);
    L.list1 = take(4 * (size_t)tiles);
    L.vlist = take(sizeof(VisitRec) * (size_t)tiles);
    L.phi_t = take(esz * (size_t)(tiles * V));
    L.tau_t = take(esz * (size_t)(tiles * V));
    L.lam_t = take(esz * (size_t)(tiles * V));
    L.r_t = take(esz * (size_t)(tiles * V));
    L.total = off;
    return true;
}

// Instances with equal gradient offsets sum into one block: chain them in
// instance order (acc_next) and number the tiles of each block's first
// instance (acc_base, monotone over all instances).  Blocks must have equal
// dims and must not overlap one another, so that one thread owns each output
// node.
bool chain_gradient_blocks(AdjLayout &L) {
    std::map<int64_t, int> first, last;     // gradient offset -> first / last instance of its chain
    std::vector<std::pair<int64_t, int64_t>> spans;
    long long acc = 0;
    for (size_t b = 0; b < L.desc_host.size(); ++b) {
        InstDesc &d = L.desc_host[b];
        d.acc_next = -1;
        d.acc_base = acc;
        auto it = first.find(d.aux_off);
        if (it == first.end()) {
            first[d.aux_off] = last[d.aux_off] = (int)b;
            acc += (long long)d.tx * d.ty * d.tz;
            spans.push_back({d.aux_off, d.aux_off + (int64_t)d.nx * d.ny * d.nz});
            continue;
        }
        const InstDesc &f = L.desc_host[(size_t)it->second];
        if (f.nx != d.nx || f.ny != d.ny || f.nz != d.nz) return false;
        L.desc_host[(size_t)last[d.aux_off]].acc_next = (int)b;
        last[d.aux_off] = (int)b;
    }
    std::sort(spans.begin(), spans.end());
    for (size_t q = 1; q < spans.size(); ++q)
        if (spans[q].first < spans[q - 1].second) return false;
    L.n_acc_tiles = acc;
    return true;
}

template <class T, int BX, int BY, int BZ>
int run_adjoint(const AdjLayout &L, const Opts &o, char *ws, const void *F, const void *phi, const int64_t *src_idx,
                int64_t n_src, const void *r, void *g, cudaStream_t st, eik_stats *stats) {
    using GG = AdjGroupGeom<BX, BY, BZ>;
    AdjParams<T> P;
    P.desc = reinterpret_cast<const InstDesc *>(ws + L.desc);
    P.B = (int)L.desc_host.size();
    P.n_tiles = (int)L.n_tiles;
    P.n_acc_tiles = (int)L.n_acc_tiles;
    P.tile_rec = reinterpret_cast<int *>(ws + L.tile_rec);
    P.tstamp = reinterpret_cast<int *>(ws + L.tstamp);
    P.list0 = reinterpret_cast<int *>(ws + L.list0);
    P.list1 = reinterpret_cast<int *>(ws + L.list1);
    P.vlist = reinterpret_cast<VisitRec *>(ws + L.vlist);
    P.phi_t = reinterpret_cast<T *>(ws + L.phi_t);
    P.tau_t = reinterpret_cast<T *>(ws + L.tau_t);
    P.lam_t = reinterpret_cast<T *>(ws + L.lam_t);
    P.r_t = reinterpret_cast<T *>(ws + L.r_t);
    P.ctl = reinterpret_cast<Ctl *>(ws + L.ctl);
    long long m = 0;
    for (const InstDesc &d : L.desc_host) m = std::max(m, (long long)d.tx + d.ty + d.tz);
    P.max_iters = o.max_iters > 0 ? o.max_iters : 64 * m + 4096;
    P.max_sweeps = 4 * (BX + BY + BZ) + 8;
    P.F = static_cast<const T *>(F);
    P.phi_in = static_cast<const T *>(phi);
    P.r_in = static_cast<const T *>(r);
    P.src_idx = reinterpret_cast<const long long *>(src_idx);
    P.n_src = n_src;
    P.g_out = static_cast<T *>(g);
    P.tkey = reinterpret_cast<unsigned *>(ws + L.tkey);
    P.inst_scale = reinterpret_cast<float *>(ws + L.inst_scale);
    P.ordered = o.order > 0.0f ? 1 : 0;
    P.order = o.order;
    P.wait_ns = o.wait_ns;
    PhaseEvents pe;
    int rc = EIK_OK;
    if (stats && (rc = pe.create())) return rc;
    pe.record(0, st);
    rc = upload_desc(const_cast<InstDesc *>(P.desc), L.desc_host, st);
    if (rc) return rc;
    DevInfo di;
    rc = device_info(di);
    if (rc) return rc;
    const unsigned span_ctas =
        (unsigned)std::max<long long>(1, std::min<long long>((L.n_tiles + kSpan - 1) / kSpan, 16ll * di.sms));
    k_adj_init<T, BX, BY, BZ><<<span_ctas, kSpanThreads, 0, st>>>(P);
    EIK_CUDA(cudaGetLastError(), "k_adj_init launch");
    if (n_src > 0) {
        k_adj_sources<T, BX, BY, BZ><<<(unsigned)((n_src + 255) / 256), 256, 0, st>>>(P);
        EIK_CUDA(cudaGetLastError(), "k_adj_sources launch");
    }
    if (P.ordered) {
        k_adj_scale<T><<<P.B, 256, 0, st>>>(P);
        EIK_CUDA(cudaGetLastError(), "k_adj_scale launch");
    }
    k_adj_list<T><<<(unsigned)std::min<long long>((L.n_tiles + 255) / 256, 4096), 256, 0, st>>>(P);
    EIK_CUDA(cudaGetLastError(), "k_adj_list launch");
    constexpr int CTA = 32 * kWarpsPerCta;
    const size_t dsm = sizeof(AdjSmem<T, BX, BY, BZ>) * GG::NG;
    // staged blocks of every group of the CTA (above the 48 KiB default for FP64 and 2D tiles)
    EIK_CUDA(cudaFuncSetAttribute((const void *)k_adj_persistent<T, BX, BY, BZ>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm),
             "dynamic shared memory attribute");
    int per_sm = 0;
    EIK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_persistent<T, BX, BY, BZ>, CTA, dsm),
             "occupancy query");
    if (!di.coop || per_sm < 1) return fail(EIK_ERR_CUDA, "the adjoint needs a cooperative launch");
    int grid = per_sm * di.sms;
    const int need = (int)((L.n_tiles + GG::NG - 1) / GG::NG);
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    pe.record(1, st);
    void *args[] = {&P};
    EIK_CUDA(cudaLaunchCooperativeKernel((const void *)k_adj_persistent<T, BX, BY, BZ>, dim3(grid), dim3(CTA), args,
                                         dsm, st),
             "cooperative launch");
    pe.record(2, st);
    const unsigned acc_ctas =
        (unsigned)std::max<long long>(1, std::min<long long>((L.n_acc_tiles + kSpan - 1) / kSpan, 16ll * di.sms));
    k_adj_output<T, BX, BY, BZ><<<acc_ctas, kSpanThreads, 0, st>>>(P);
    EIK_CUDA(cudaGetLastError(), "k_adj_output launch");
    pe.record(3, st);
    if (stats) return finish_stats(P.ctl, st, stats, &pe);
    return EIK_OK;
}

int adjoint_impl(int64_t B, const eik_grid *grids, const void *F, const int64_t *F_offsets, const void *phi,
                 const int64_t *phi_offsets, const int64_t *src_idx, const int64_t *src_offsets, const void *r,
                 void *g, const int64_t *g_offsets, void *ws, size_t ws_bytes, void *stream, const eik_options *opt,
                 eik_stats *stats) {
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (B < 1 || B > (1ll << 24)) return fail(EIK_ERR_ARG, "batch size must be in [1, 2^24]");
    if (!grids || !F_offsets || !phi_offsets || !src_offsets || !g_offsets)
        return fail(EIK_ERR_ARG, "grids and offset arrays must be non-NULL");
    Opts o;
    if (!read_opts(opt, B, grids, o)) return fail(EIK_ERR_ARG, "invalid options");
    // the adjoint's own defaults (measured on the 192^3 16-shot tomography): larger tiles and a
    // wider window than the forward, since its order is static and known in advance
    bool all2d = true;
    for (int64_t b = 0; b < B; ++b) all2d = all2d && grids[b].nz == 1;
    if (!opt || opt->tile == EIK_TILE_AUTO) o.tile = all2d ? EIK_TILE_16x16x1 : EIK_TILE_8x8x8;
    if (!opt || opt->order == 0.0f) o.order = kDefaultAdjointOrder;
    AdjLayout L;
    std::string why;
    if (!make_adj_layout(B, grids, o, L, &why)) return fail(EIK_ERR_ARG, "%s", why.c_str());
    if (!ws) return fail(EIK_ERR_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(EIK_ERR_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < L.total) return fail(EIK_ERR_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
    if (!F || !phi || !r || !g) return fail(EIK_ERR_ARG, "F, phi, r and g must be non-NULL");
    if (src_offsets[0] != 0) return fail(EIK_ERR_ARG, "src_offsets[0] must be 0");
    for (int64_t b = 0; b < B; ++b) {
        if (src_offsets[b + 1] < src_offsets[b]) return fail(EIK_ERR_ARG, "src_offsets must be non-decreasing");
        if (F_offsets[b] < 0 || phi_offsets[b] < 0 || g_offsets[b] < 0) return fail(EIK_ERR_ARG, "offsets must be >= 0");
        InstDesc &d = L.desc_host[(size_t)b];
        d.in_off = F_offsets[b];
        d.out_off = phi_offsets[b];
        d.aux_off = g_offsets[b];
        d.src_begin = src_offsets[b];
        d.src_end = src_offsets[b + 1];
    }
    if (!chain_gradient_blocks(L)) return fail(EIK_ERR_ARG, "gradient blocks must be equal (same offset and dims) or disjoint");
    const int64_t n_src = src_offsets[B];
    if (n_src > 0 && !src_idx) return fail(EIK_ERR_ARG, "src_idx must be non-NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(ws);
#define EIK_ADJ_DISPATCH(T)                                                                                       \
    switch (o.tile) {                                                                                             \
        case EIK_TILE_4x4x4: return run_adjoint<T, 4, 4, 4>(L, o, w, F, phi, src_idx, n_src, r, g, st, stats);    \
        case EIK_TILE_8x8x4: return run_adjoint<T, 8, 8, 4>(L, o, w, F, phi, src_idx, n_src, r, g, st, stats);    \
        case EIK_TILE_16x16x1: return run_adjoint<T, 16, 16, 1>(L, o, w, F, phi, src_idx, n_src, r, g, st, stats); \
        case EIK_TILE_8x4x4: return run_adjoint<T, 8, 4, 4>(L, o, w, F, phi, src_idx, n_src, r, g, st, stats);    \
        case EIK_TILE_8x8x1: return run_adjoint<T, 8, 8, 1>(L, o, w, F, phi, src_idx, n_src, r, g, st, stats);    \
        default: return run_adjoint<T, 8, 8, 8>(L, o, w, F, phi, src_idx, n_src, r, g, st, stats);                \
    }
    if (o.precision == EIK_FP64) { EIK_ADJ_DISPATCH(double) }
    EIK_ADJ_DISPATCH(float)
#undef EIK_ADJ_DISPATCH
}

// ---------------------------------------------------------------- no-allocation variant
// Fixed scratch for eik_solve_noalloc: a file-scope device array, so a caller
// that may not allocate device memory still gets a workspace.  Every device
// that loads this library holds these bytes until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (the host-side
// name of the array is not a device address).  It is looked up again on every
// call made outside stream capture -- a cheap host-side query once the module
// is loaded, which also picks up a new address after cudaDeviceReset() -- and
// remembered per device for calls made while `stream` is being captured, which
// need an earlier uncaptured call on that device.
int noalloc_scratch(cudaStream_t stream, void **out) {
    int dev = -1;
    EIK_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(EIK_ERR_ARG, "device index %d out of range", dev);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    EIK_CUDA(cudaStreamIsCapturing(stream, &cap), "cudaStreamIsCapturing");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        EIK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(scratch)");
        g_scratch_addr[dev] = p;
    } else if (!g_scratch_addr[dev]) {
        return fail(EIK_ERR_ARG, "eik_solve_noalloc: make one call on this device outside stream capture first");
    }
    *out = g_scratch_addr[dev];
    return EIK_OK;
}

}  // namespace

extern "C" {

size_t eik_workspace_size_batched(int64_t B, const eik_grid *grids, const eik_options *opt) {
    if (B < 1 || !grids) return 0;
    Opts o;
    if (!read_opts(opt, B, grids, o)) return 0;
    Layout L;
    if (!make_layout(B, grids, o, L, nullptr)) return 0;
    return L.total;
}

size_t eik_workspace_size(const eik_grid *grid, const eik_options *opt) {
    return eik_workspace_size_batched(1, grid, opt);
}

int eik_solve(const eik_grid *grid, const void *F, const int64_t *src_idx, const void *src_val, int64_t n_src,
              void *phi, void *workspace, size_t workspace_bytes, void *stream, const eik_options *opt,
              eik_stats *stats) {
    if (n_src < 0) return fail(EIK_ERR_ARG, "n_src must be >= 0");
    const int64_t zero = 0;
    const int64_t so[2] = {0, n_src};
    return solve_impl(1, grid, F, &zero, src_idx, src_val, so, phi, &zero, workspace, workspace_bytes, stream, opt,
                      stats);
}

int eik_solve_batched(int64_t B, const eik_grid *grids, const void *F_packed, const int64_t *F_offsets,
                      const int64_t *src_idx, const void *src_val, const int64_t *src_offsets, void *phi_packed,
                      const int64_t *phi_offsets, void *workspace, size_t workspace_bytes, void *stream,
                      const eik_options *opt, eik_stats *stats) {
    if (!F_offsets || !src_offsets || !phi_offsets) return fail(EIK_ERR_ARG, "offset arrays must be non-NULL");
    return solve_impl(B, grids, F_packed, F_offsets, src_idx, src_val, src_offsets, phi_packed, phi_offsets,
                      workspace, workspace_bytes, stream, opt, stats);
}

int eik_solve_noalloc(const eik_grid *grid, const void *F, const int64_t *src_idx, const void *src_val,
                      int64_t n_src, void *phi, void *stream, const eik_options *opt, eik_stats *stats) {
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n_src < 0) return fail(EIK_ERR_ARG, "n_src must be >= 0");
    const size_t need = eik_workspace_size(grid, opt);
    if (need == 0) return fail(EIK_ERR_ARG, "invalid grid or options");
    if (need > kNoAllocScratchBytes)
        return fail(EIK_ERR_ARG,
                    "grid needs %zu bytes of scratch but the static scratch of eik_solve_noalloc holds %zu; "
                    "call eik_solve with a caller-provided workspace instead",
                    need, kNoAllocScratchBytes);
    void *scratch = nullptr;
    const int rc = noalloc_scratch(static_cast<cudaStream_t>(stream), &scratch);
    if (rc) return rc;
    // the solve initialises every part of the workspace it reads (control
    // block, per-tile state, keys, lists), so stale contents of the shared
    // array from an earlier call do not matter
    return eik_solve(grid, F, src_idx, src_val, n_src, phi, scratch, kNoAllocScratchBytes, stream, opt, stats);
}

int eik_backtrace(const eik_grid *grid, int precision, const void *phi, const int64_t *start_idx, int64_t n_paths,
                  int64_t max_len, int64_t *path, int64_t *len, void *stream) {
    if (!grid || !phi) return fail(EIK_ERR_ARG, "null grid or phi");
    const eik_grid &g = *grid;
    if (g.nx < 1 || g.ny < 1 || g.nz < 1 || g.nx > (1ll << 30) || g.ny > (1ll << 30) || g.nz > (1ll << 30))
        return fail(EIK_ERR_ARG, "dims must be in [1, 2^30]");
    if (!(g.h > 0.0) || !(g.h < 1e300) || !spacing_ok(g.hy) || !spacing_ok(g.hz))
        return fail(EIK_ERR_ARG, "h must be finite and > 0; hy, hz 0 or finite and > 0");
    if (precision != EIK_FP32 && precision != EIK_FP64) return fail(EIK_ERR_ARG, "unknown precision");
    if (n_paths < 0 || n_paths > (1ll << 28)) return fail(EIK_ERR_ARG, "n_paths must be in [0, 2^28]");
    if (max_len < 1 || max_len > (1ll << 34) / std::max<int64_t>(n_paths, 1))
        return fail(EIK_ERR_ARG, "max_len must be >= 1 and n_paths * max_len <= 2^34");
    if (n_paths == 0) return EIK_OK;
    if (!start_idx || !path || !len) return fail(EIK_ERR_ARG, "null start_idx, path or len");
    BacktraceConst bc;
    const double hx = g.h, hy = spacing_y(g), hz = spacing_z(g);
    for (int l = 0; l < 26; ++l) {
        const int c = l < 13 ? l : l + 1;
        const double ox = (c % 3 - 1) * hx, oy = ((c / 3) % 3 - 1) * hy, oz = (c / 9 - 1) * hz;
        const double sq = ox * ox + oy * oy + oz * oz;
        bc.inv_len[l] = 1.0 / std::sqrt(sq);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned blocks = (unsigned)((n_paths * 32 + 255) / 256);
    const long long *si = reinterpret_cast<const long long *>(start_idx);
    long long *po = reinterpret_cast<long long *>(path), *lo = reinterpret_cast<long long *>(len);
    if (precision == EIK_FP64)
        k_backtrace<double><<<blocks, 256, 0, st>>>(static_cast<const double *>(phi), (int)g.nx, (int)g.ny, (int)g.nz,
                                                    bc, si, n_paths, max_len, po, lo);
    else
        k_backtrace<float><<<blocks, 256, 0, st>>>(static_cast<const float *>(phi), (int)g.nx, (int)g.ny, (int)g.nz,
                                                   bc, si, n_paths, max_len, po, lo);
    EIK_CUDA(cudaGetLastError(), "k_backtrace launch");
    return EIK_OK;
}

int eik_set_trace(void *device_buffer, int64_t capacity) {
    if (capacity < 0 || (device_buffer && capacity < 1)) return fail(EIK_ERR_ARG, "invalid trace capacity");
    if (device_buffer && reinterpret_cast<uintptr_t>(device_buffer) % 8) return fail(EIK_ERR_ARG, "trace buffer must be 8-byte aligned");
    unsigned long long *p = static_cast<unsigned long long *>(device_buffer);
    long long cap = device_buffer ? (long long)capacity : 0;
    EIK_CUDA(cudaMemcpyToSymbol(g_trace_buf, &p, sizeof(p)), "cudaMemcpyToSymbol(trace)");
    EIK_CUDA(cudaMemcpyToSymbol(g_trace_cap, &cap, sizeof(cap)), "cudaMemcpyToSymbol(trace)");
    return EIK_OK;
}

size_t eik_adjoint_workspace_size_batched(int64_t B, const eik_grid *grids, const eik_options *opt) {
    if (B < 1 || !grids) return 0;
    Opts o;
    if (!read_opts(opt, B, grids, o)) return 0;
    bool all2d = true;
    for (int64_t b = 0; b < B; ++b) all2d = all2d && grids[b].nz == 1;
    if (!opt || opt->tile == EIK_TILE_AUTO) o.tile = all2d ? EIK_TILE_16x16x1 : EIK_TILE_8x8x8;
    AdjLayout L;
    if (!make_adj_layout(B, grids, o, L, nullptr)) return 0;
    return L.total;
}

int eik_adjoint_batched(int64_t B, const eik_grid *grids, const void *F_packed, const int64_t *F_offsets,
                        const void *phi_packed, const int64_t *phi_offsets, const int64_t *src_idx,
                        const int64_t *src_offsets, const void *r_packed, void *g_packed, const int64_t *g_offsets,
                        void *workspace, size_t workspace_bytes, void *stream, const eik_options *opt,
                        eik_stats *stats) {
    return adjoint_impl(B, grids, F_packed, F_offsets, phi_packed, phi_offsets, src_idx, src_offsets, r_packed,
                        g_packed, g_offsets, workspace, workspace_bytes, stream, opt, stats);
}

int eik_adjoint(const eik_grid *grid, const void *F, const void *phi, const int64_t *src_idx, int64_t n_src,
                const void *r, void *g, void *workspace, size_t workspace_bytes, void *stream,
                const eik_options *opt, eik_stats *stats) {
    if (n_src < 0) return fail(EIK_ERR_ARG, "n_src must be >= 0");
    const int64_t zero = 0;
    const int64_t so[2] = {0, n_src};
    return adjoint_impl(1, grid, F, &zero, phi, &zero, src_idx, so, r, g, &zero, workspace, workspace_bytes, stream,
                        opt, stats);
}

const char *eik_last_error(void) { return g_err.c_str(); }

const char *eik_version(void) { return "eikonal-b300 0.1 (sm_103a)"; }

}  // extern "C"
