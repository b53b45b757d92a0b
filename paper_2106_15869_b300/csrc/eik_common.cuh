// eik_common.cuh -- shared device definitions of the iFIM CUDA path (sm_103a).
//
// Data layout in HBM (per solve, inside the caller's workspace):
//   phi_t, tau_t   bricked: tile g occupies [g*V, (g+1)*V), V = BX*BY*BZ nodes,
//                  x fastest inside the tile; tiles of an instance are ordered
//                  (tz, ty, tx) and instances follow each other (tile_base).
//                  Nodes of a boundary tile that lie outside the grid carry
//                  tau = +inf and phi = +inf forever.
//   tau            h / F per node (+inf where F == 0, eq. 8 barrier); a fixed
//                  source node carries tau = +inf as well: its local solve
//                  then gives NaN or +inf, never a value below its own, so
//                  the sweeps need no per-node test (measured: the test in the
//                  sweep cost 5-6 % of the loop on every 3D workload).
//   tstate         per tile: 0 Distant, 1 Active, 2 Source (Algorithm 2 sets,
//                  taken at tile granularity)
//   tstamp         per tile: remedy-list membership stamp (iteration + 1)
//   list0/list1    tile-id lists (Active or Remedy), ping-pong by iteration
//   Ctl            counters, barrier word, flags and statistics
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace eik {

constexpr int kMaxInstPerLaunch = 128;       // descriptors passed by value per launch
// default bound on every device wait (2 s); a call may set another (eik_options.wait_limit_us)
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// device flag bits (eik_stats.device_flags)
constexpr int kFlagCap = 1;          // iteration cap reached
constexpr int kFlagTimeout = 2;      // a bounded wait gave up
constexpr int kFlagBadSource = 4;    // a source index outside its grid (ignored)
constexpr int kFlagOverflow = 8;     // a list push beyond capacity (internal error)
constexpr int kFlagDebugIndex = 16;  // EIK_DEBUG builds: a tile id read from a list or queue out of range
constexpr int kFlagDebugNaN = 32;    // EIK_DEBUG builds: a NaN written to phi or lambda

// Debug build (compiled with -DEIK_DEBUG, libeikonal_debug.so): every tile id
// read from a list, a visit record or the work queue is checked against the
// tile count before use, and every value written back to phi or lambda is
// checked for NaN.  A failed check raises a device flag (reported by the call
// as EIK_ERR_DEVICE) and the access is skipped; nothing traps.  In the release
// build the checks compile to nothing.
#ifdef EIK_DEBUG
constexpr bool kDebug = true;
#else
constexpr bool kDebug = false;
#endif

enum TileState : int { kDistant = 0, kActive = 1, kSource = 2 };

struct InstDesc {
    int32_t nx, ny, nz;
    int32_t acc_next;             // adjoint: next instance summing into the same gradient block (-1: none)
    int32_t tx, ty, tz, pad1;     // tiles per axis
    int64_t tile_base;            // first global tile id of this instance
    int64_t in_off;               // element offset of F (and of r in the adjoint)
    int64_t out_off;              // element offset of phi (and of g in the adjoint)
    int64_t src_begin, src_end;   // entries of the packed source arrays
    double h;
    int64_t aux_off;              // element offset of the adjoint's gradient output
    int64_t acc_base;             // adjoint: tiles of the gradient blocks' first instances before this one
};

// Partial slowness statistics of a slice of an instance's tiles (key-scale reduction).
struct ScalePart {
    double sum, cnt;
};

struct DescChunk {                // by-value kernel parameter (capture-safe upload)
    InstDesc d[kMaxInstPerLaunch];
    int first, count;
};

struct Ctl {
    unsigned long long bar;       // grid-barrier arrivals (monotone within a launch)
    int abort;                    // a barrier wait timed out: every block leaves
    int flags;                    // kFlag* bits
    int cnt[3];                   // Step-2 list sizes, slot = iteration % 3
    int rcnt[3];                  // Step-3 list sizes
    unsigned kmin[3];             // Step-2 smallest key listed for iteration it (slot it % 3)
    unsigned rkmin[3];            // Step-3 smallest key listed for iteration r
    int nproc[4];                 // tiles visited (not deferred) in iteration it (slot it % 4)
    int grab[3], rgrab[3];        // latency mode: list entries taken so far in iteration it (slot it % 3)
    float win[2];                 // bucket width of the host-loop schedule, by iteration parity
    long long iters_update, iters_remedy;
    long long tiles_update, tiles_flagged, tiles_remedy, sweeps, tiles_deferred;
    unsigned long long q_head, q_tail;   // work-queue positions (asynchronous schedule)
    int q_pending;                       // tiles queued or being visited in the current phase
    int q_stop;                          // the visit cap was reached: every warp leaves the phase
    long long q_visits;                  // visits in the current phase (cap check)
    int vcnt[3], vgrab[3];               // two-phase Step-2 iterations: kept tiles listed / taken, slot it % 3
    int rvcnt[3], rvgrab[3];             // the same for Step 3
};
static_assert(sizeof(Ctl) <= 256, "the control block is zeroed by 64 threads");

// debug build: true (and the flag raised) when tile id g is outside [0, n)
__device__ __forceinline__ bool dbg_bad_tile(Ctl *ctl, long long g, long long n) {
    if constexpr (kDebug) {
        if (g < 0 || g >= n) {
            atomicOr(&ctl->flags, kFlagDebugIndex);
            return true;
        }
    }
    return false;
}
// debug build: raise the flag when a value written back is NaN
template <class T>
__device__ __forceinline__ void dbg_nan(Ctl *ctl, T v) {
    if constexpr (kDebug) {
        if (v != v) atomicOr(&ctl->flags, kFlagDebugNaN);
    }
}

// Ordered-float encoding for atomicMin on keys: monotone as unsigned.
__device__ __forceinline__ unsigned key_enc(float k) {
    const unsigned b = __float_as_uint(k);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_dec(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
constexpr unsigned kKeyInf = 0xff800000u;   // key_enc(+inf)

// Encoded key of value v for an instance with key scale sc (1/delta).  A
// scale of 0 marks an instance that is not ordered: all its keys are 0, so
// its listed tiles are always inside the window.
__device__ __forceinline__ unsigned scaled_key(float v, float sc) { return key_enc(sc > 0.0f ? v * sc : 0.0f); }

// ----------------------------------------------------------------- helpers
template <class T> struct Num;
template <> struct Num<float> {
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
};
template <> struct Num<double> {
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
};

__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float vsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double vsqrt(double a) { return sqrt(a); }

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ double ld_volatile_d(const double *p) { return *(const volatile double *)p; }
__device__ __forceinline__ float ld_volatile_f(const float *p) { return *(const volatile float *)p; }

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }
__device__ __forceinline__ unsigned ld_volatile_u(const unsigned *p) { return *(const volatile unsigned *)p; }
// Bucket width of the ordered schedule for the next iteration (the same in
// every CTA).  It doubles while an iteration visits less than 1/16 of its
// list and fewer tiles than half the thread groups of the launch (most of the
// list waits, and the GPU would idle: keys spread over many buckets, e.g.
// behind slow walls), and halves back toward one unit once more than half of
// a list is visited.  Widths are in key units (order * tile-crossing times).
__device__ __forceinline__ float adapt_window(float w, int visited, int listed, int groups, int warps) {
    (void)warps;
    if (listed <= 0) return w;
    if (16 * visited < listed && 2 * visited < groups) w *= 2.0f;
    else if (2 * visited > listed) w = fmaxf(1.0f, 0.5f * w);
    return fminf(w, 1e30f);
}

__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exact root of eq. (6) given the per-axis upwind minima and tau = h/F:
//   sum_d ((u - a_d)^+)^2 = tau^2, a1 <= a2 <= a3 sorted.
// One-sided u = a1 + tau while u <= a2; two-sided while u <= a3; else
// three-sided.  The roots are formed relative to a1 (d2 = a2 - a1,
// d3 = a3 - a1) so that no large sums cancel in FP32:
//   two-sided   u = a1 + (d2 + sqrt(2 tau^2 - d2^2)) / 2
//   three-sided u = a1 + (d2 + d3 + sqrt(3 tau^2 - d2^2 - d3^2 - (d3 - d2)^2)) / 3
// The thresholds are the validity conditions of the "^+" equation (Alg 1.1
// and Alg 1.3 print others).  a1 = +inf or tau = +inf yields +inf.
template <class T>
__device__ __forceinline__ T local_solve(T ax, T ay, T az, T tau) {
    const T lo = vmin(ax, ay), hi = vmax(ax, ay);
    const T a1 = vmin(lo, az);
    const T a3 = vmax(hi, az);
    const T a2 = vmax(lo, vmin(hi, az));
    T u = a1 + tau;
    if (u <= a2) return u;
    const T d2 = a2 - a1;
    u = a1 + T(0.5) * (d2 + vsqrt(T(2) * tau * tau - d2 * d2));
    if (u <= a3) return u;
    const T d3 = a3 - a1, d32 = d3 - d2;
    T disc = T(3) * tau * tau - (d2 * d2 + d3 * d3 + d32 * d32);
    disc = vmax(disc, T(0));
    return a1 + (d2 + d3 + vsqrt(disc)) * (T(1) / T(3));
}

// FP32 form for the relaxation sweeps, where the latency of one root is on the
// critical path of the wavefront: the same cascade, but the three candidate
// roots are formed at once (their square roots overlap) and then selected,
// and the square root is x * rsqrt(x) (a few ulp; the FP32 solve is held to
// 1e-4 of max(phi)).  A candidate whose branch is not taken may be NaN, inf or
// (from a negative discriminant) a root of the clamped argument; it is never
// selected: a negative two-sided discriminant means d2 > sqrt(2) tau, so the
// one-sided root lies below a2, and a negative three-sided one means the
// two-sided root lies below a3.  The three-sided discriminant uses
// d2^2 + d3^2 + (d3 - d2)^2 = 2 (d2^2 + d3^2 - d2 d3).
//
// The reciprocal root is the PTX approximate instruction with flush to zero:
// without the input range handling that rsqrtf carries for subnormal
// arguments, the sweeps run 6-8 % faster on B300 (every 3D workload; same
// results to the last printed digit of the error).  The argument is clamped to
// at least 1e-30 (one max instead of a compare and a select): a discriminant at
// or below it gives 1e-15, far under any arrival-time spacing, and no flushed
// subnormal reaches the product as 0 * inf.
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    x = fmaxf(x, 1e-30f);
    return x * rsqrt_ftz(x);
}

__device__ __forceinline__ float local_solve_fast(float ax, float ay, float az, float tau) {
    const float lo = fminf(ax, ay), hi = fmaxf(ax, ay);
    const float a1 = fminf(lo, az);
    const float a3 = fmaxf(hi, az);
    const float a2 = fmaxf(lo, fminf(hi, az));
    const float u1 = a1 + tau;
    const float d2 = a2 - a1, d3 = a3 - a1;
    const float t2 = tau * tau;
    const float u2 = fmaf(0.5f, d2 + sqrt_approx(fmaf(-d2, d2, t2 + t2)), a1);
    const float q = fmaf(-d2, d3, fmaf(d3, d3, d2 * d2));
    const float u3 = fmaf(d2 + d3 + sqrt_approx(fmaf(-2.0f, q, 3.0f * t2)), 1.0f / 3.0f, a1);
    return u1 <= a2 ? u1 : (u2 <= a3 ? u2 : u3);
}

// the root used by the relaxation sweeps: fast form in FP32, exact form in FP64
__device__ __forceinline__ float sweep_solve(float ax, float ay, float az, float tau) {
    return local_solve_fast(ax, ay, az, tau);
}
__device__ __forceinline__ double sweep_solve(double ax, double ay, double az, double tau) {
    return local_solve<double>(ax, ay, az, tau);
}

// Unequal spacings (eq. 5/6 with dx, dy, dz; Alg 1.2).  With tau = dx / F and
// axis weights c_d = (dx / h_d)^2 (c_x = 1) the equation is
//   sum_d c_d ((u - a_d)^+)^2 = tau^2,
// solved by the same prefix cascade over the minima sorted by value, each
// minimum carrying its weight (d2 = a2 - a1, d3 = a3 - a1, C = c1 + c2 + c3):
//   one-sided   u = a1 + tau / sqrt(c1)                                       valid iff u <= a2
//   two-sided   u = a1 + (c2 d2 + sqrt((c1 + c2) tau^2 - c1 c2 d2^2)) / (c1 + c2)   valid iff u <= a3
//   three-sided u = a1 + (c2 d2 + c3 d3 + sqrt(C tau^2 - c1 c2 d2^2 - c1 c3 d3^2 - c2 c3 (d3 - d2)^2)) / C
// The weights are per call (every grid of a call has the same spacing ratios).
template <class T>
struct Metric {
    T cy, cz;     // (dx / dy)^2, (dx / dz)^2
    int aniso;    // 0: equal spacings, the isotropic cascade
    T r_xy, r_xz, r_yz, r_xyz;   // 1 / (1 + cy), 1 / (1 + cz), 1 / (cy + cz), 1 / (1 + cy + cz)
};

// compare-exchange of (minimum, weight) pairs by minimum
template <class T>
__device__ __forceinline__ void cx_pair(T &a, T &c, T &b, T &e) {
    const bool sw = b < a;
    const T a0 = a, c0 = c;
    a = sw ? b : a; c = sw ? e : c;
    b = sw ? a0 : b; e = sw ? c0 : e;
}

template <class T>
__device__ __forceinline__ T local_solve_w(T ax, T ay, T az, T tau, T cy, T cz) {
    T a1 = ax, c1 = T(1), a2 = ay, c2 = cy, a3 = az, c3 = cz;
    cx_pair(a1, c1, a2, c2);
    cx_pair(a2, c2, a3, c3);
    cx_pair(a1, c1, a2, c2);
    T u = a1 + tau / vsqrt(c1);
    if (u <= a2) return u;
    const T d2 = a2 - a1, t2 = tau * tau, C2 = c1 + c2;
    u = a1 + (c2 * d2 + vsqrt(vmax(C2 * t2 - c1 * c2 * d2 * d2, T(0)))) / C2;
    if (u <= a3) return u;
    const T d3 = a3 - a1, d32 = d3 - d2, C3 = C2 + c3;
    T disc = C3 * t2 - (c1 * c2 * d2 * d2 + c1 * c3 * d3 * d3 + c2 * c3 * d32 * d32);
    disc = vmax(disc, T(0));
    return a1 + (c2 * d2 + c3 * d3 + vsqrt(disc)) / C3;
}

// FP32 sweep form of local_solve_w: the three candidate roots at once, then
// the selection (as local_solve_fast).  The weight sums C2 and C3 take one of
// four values per call, whose reciprocals the call provides: the two-sided sum
// is fixed by the weight left out (c3), so no root divides.
__device__ __forceinline__ float local_solve_fast_w(float ax, float ay, float az, float tau, const Metric<float> &mt) {
    float a1 = ax, c1 = 1.0f, a2 = ay, c2 = mt.cy, a3 = az, c3 = mt.cz;
    cx_pair(a1, c1, a2, c2);
    cx_pair(a2, c2, a3, c3);
    cx_pair(a1, c1, a2, c2);
    const float rC2 = c3 == 1.0f ? mt.r_yz : (c3 == mt.cy ? mt.r_xz : mt.r_xy);
    const float t2 = tau * tau, C2 = c1 + c2, C3 = C2 + c3;
    const float d2 = a2 - a1, d3 = a3 - a1, d32 = d3 - d2;
    const float u1 = a1 + tau * rsqrt_ftz(c1);   // c1 is 1, (dx/dy)^2 or (dx/dz)^2
    const float u2 = a1 + (c2 * d2 + sqrt_approx(C2 * t2 - c1 * c2 * d2 * d2)) * rC2;
    const float u3 =
        a1 + (c2 * d2 + c3 * d3 + sqrt_approx(C3 * t2 - (c1 * c2 * d2 * d2 + c1 * c3 * d3 * d3 + c2 * c3 * d32 * d32))) *
                 mt.r_xyz;
    return u1 <= a2 ? u1 : (u2 <= a3 ? u2 : u3);
}

__device__ __forceinline__ float sweep_solve_w(float ax, float ay, float az, float tau, const Metric<float> &mt) {
    return local_solve_fast_w(ax, ay, az, tau, mt);
}
__device__ __forceinline__ double sweep_solve_w(double ax, double ay, double az, double tau, const Metric<double> &mt) {
    return local_solve_w<double>(ax, ay, az, tau, mt.cy, mt.cz);
}

// The root every relaxation uses: isotropic cascade, or the weighted one.
// The same with the spacing case fixed at compile time: the sweeps of the
// group passes select it once per visit, not once per node.
template <bool ANISO, class T>
__device__ __forceinline__ T node_solve_fixed(T ax, T ay, T az, T tau, const Metric<T> &mt) {
    if constexpr (ANISO)
        return sweep_solve_w(ax, ay, az, tau, mt);
    else
        return sweep_solve(ax, ay, az, tau);
}
template <class T>
__device__ __forceinline__ T node_solve(T ax, T ay, T az, T tau, const Metric<T> &mt) {
    return mt.aniso ? sweep_solve_w(ax, ay, az, tau, mt) : sweep_solve(ax, ay, az, tau);
}

// Device-wide barrier for a cooperative launch.  Every wait is bounded by
// limit_ns of %globaltimer; on a timeout the block raises ctl->abort and every
// block leaves at its next barrier.  Returns false when the launch must stop.
__device__ __forceinline__ bool grid_sync(Ctl *ctl, unsigned long long &target, unsigned long long limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        __threadfence();
        atomicAdd(&ctl->bar, 1ull);
        const unsigned long long t0 = globaltimer();
        int ok = 1;
        while (ld_acquire(&ctl->bar) < target) {
            if (ld_volatile(&ctl->abort)) { ok = 0; break; }
            if (globaltimer() - t0 > limit_ns) {
                atomicOr(&ctl->flags, kFlagTimeout);
                atomicExch(&ctl->abort, 1);
                ok = 0;
                break;
            }
            __nanosleep(40);
        }
        __threadfence();
        if (ld_volatile(&ctl->abort)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// binary search: instance whose [tile_base, next tile_base) holds tile g
__device__ __forceinline__ int find_inst_by_tile(const InstDesc *desc, int B, long long g) {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (desc[mid].tile_base <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// binary search over the adjoint's gradient blocks: the last instance with
// acc_base <= a, which is the first instance of the block holding tile a of
// the blocks' tile space (acc_base grows only across first instances).
__device__ __forceinline__ int find_inst_by_acc(const InstDesc *desc, int B, long long a) {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (desc[mid].acc_base <= a) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// binary search: instance whose [src_begin, src_end) holds source entry s
__device__ __forceinline__ int find_inst_by_src(const InstDesc *desc, int B, long long s) {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (desc[mid].src_begin <= s) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace eik
