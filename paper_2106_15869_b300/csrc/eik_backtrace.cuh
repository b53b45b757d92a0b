// eik_backtrace.cuh -- shortest-path back-trace on a phi map (sm_103a).
//
// The application of Example 4 (Sec. 4.1): from a destination node, descend
// the arrival-time map to the source.  The paper names gradient descent on
// phi without the discrete rule; this is the steepest descent on the grid
// graph: the next node is the neighbour among the 26 (8 in 2D) adjacent
// nodes with the smallest slope (phi[nb] - phi[cur]) / |x_nb - x_cur|
// (physical distance with spacings dx, dy, dz) among those with
// phi[nb] < phi[cur]; ties go to the lower flat index.  The path ends at a
// node without a lower neighbour (a source, since every other reachable node
// has a face neighbour with a smaller value) or when the path buffer is full.
//
// One warp per path: lane l < 26 owns one neighbour offset, loads it, forms
// its slope in double (phi values of either precision convert exactly; the
// slope is a rounded subtraction then a rounded product with the offset's
// 1/length, so the decision is the same as any IEEE double evaluation of the
// rule), and the warp takes the lexicographic (slope, index) minimum.
#pragma once

#include "eik_common.cuh"

namespace eik {

struct BacktraceConst {
    double inv_len[26];         // 1 / |offset| of neighbour slot l (physical units)
};

// neighbour slot l (0..25) -> offsets in -1..1, the centre skipped
__device__ __forceinline__ void bt_offset(int l, int &di, int &dj, int &dk) {
    const int c = l < 13 ? l : l + 1;
    di = c % 3 - 1;
    dj = (c / 3) % 3 - 1;
    dk = c / 9 - 1;
}

template <class T>
__global__ void k_backtrace(const T *__restrict__ phi, int nx, int ny, int nz, BacktraceConst bc,
                            const long long *__restrict__ start, long long n_paths, long long max_len,
                            long long *__restrict__ path, long long *__restrict__ len) {
    const long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= n_paths) return;                                   // warp-uniform
    const int lane = threadIdx.x & 31;
    long long *row = path + q * max_len;
    for (long long t = lane; t < max_len; t += 32) row[t] = -1;
    const long long N = (long long)nx * ny * nz;
    long long cur = start[q];
    if (cur < 0 || cur >= N) {
        if (lane == 0) len[q] = -1;
        return;
    }
    double pc = (double)phi[cur];
    long long n = 0;
    if (pc < (double)Num<T>::inf()) {
        if (lane == 0) row[0] = cur;
        n = 1;
        int di = 0, dj = 0, dk = 0;
        if (lane < 26) bt_offset(lane, di, dj, dk);
        const double il = lane < 26 ? bc.inv_len[lane] : 0.0;
        while (n < max_len) {
            const int i = (int)(cur % nx), j = (int)((cur / nx) % ny), k = (int)(cur / ((long long)nx * ny));
            const int a = i + di, b = j + dj, c = k + dk;
            double slope = __longlong_as_double(0x7ff0000000000000ll);   // +inf: no candidate
            long long nb = 0x7fffffffffffffffll;
            double pn = 0.0;
            if (lane < 26 && a >= 0 && b >= 0 && c >= 0 && a < nx && b < ny && c < nz) {
                const long long m = ((long long)c * ny + b) * nx + a;
                pn = (double)__ldg(phi + m);
                if (pn < pc) {
                    slope = __dmul_rn(__dsub_rn(pn, pc), il);
                    nb = m;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double s2 = __shfl_xor_sync(kFull, slope, o);
                const long long n2 = __shfl_xor_sync(kFull, nb, o);
                const double p2 = __shfl_xor_sync(kFull, pn, o);
                if (s2 < slope || (s2 == slope && n2 < nb)) { slope = s2; nb = n2; pn = p2; }
            }
            if (nb == 0x7fffffffffffffffll) break;                    // no lower neighbour (warp-uniform)
            cur = nb;
            pc = pn;
            if (lane == 0) row[n] = cur;
            ++n;
        }
    }
    if (lane == 0) len[q] = n;
}

}  // namespace eik
