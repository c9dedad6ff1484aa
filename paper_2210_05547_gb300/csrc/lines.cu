// Batched compact staggered line operators (Sec. 3.1): y = A^{-1} (B x) along grid lines.
//
// GB300 retires two FP64 FMAs per clock per SM, so one warp-wide FP64 instruction occupies an
// SM sub-partition for 64 cycles: a Thomas sweep of one 2049-point line run by a single thread
// takes about a millisecond. The work is therefore spread over segments of each line.
//
// Every line is cut into `nseg` segments that live in the same thread block. Thread k:
//   1. runs the forward recurrence d_r = (rhs_r - l_r d_{r-1}) / piv_r from W rows before its
//      segment (starting from 0 there; exact when that start is row 0) and stores d_r for its own
//      rows in `tmp`;
//   2. after a barrier, runs the back substitution y_r = d_r - c'_r y_{r+1} from W rows past its
//      segment end (starting from y = d there; exact at the last row), reading the forward values
//      its neighbours stored, and writes its own rows.
// The factors satisfy |l_r / piv_r| <= 1/3 and |c'_r| <= 1/3, so the history dropped at the
// start of either recurrence is scaled by at most 3^-W: W = 40 (interpolation, alpha = 3/10) and
// W = 26 (derivative, alpha = 9/62, factor <= 0.148) leave it below 1e-19 of the values, under
// FP64 rounding. Each segment reads only values written before the barrier by threads of its own
// block, so results are deterministic.
#include "internal.h"

namespace hyp {
namespace {

__device__ __forceinline__ double closure_rhs(const LineOp& op, const double* __restrict__ in,
                                              long long ies, int r, double wall) {
    int c = 0;
    while (op.crow[c] != r) ++c;
    double v = op.gw[c] * wall;
    const double* p = in + (long long)op.cstart[c] * ies;
    for (int k = 0; k < op.cnum[c]; ++k) v += op.cw[c][k] * p[(long long)k * ies];
    return v;
}

__global__ void __launch_bounds__(LINE_BLOCK) k_lines(const LineJob* __restrict__ jobs,
                                               const double* __restrict__ U) {
    const LineJob& J = jobs[blockIdx.y];
    const int nseg = J.nseg;
    const int lpb = blockDim.x / nseg;                  // lines per block
    const int seg = threadIdx.x / lpb;
    const int line = blockIdx.x * lpb + (threadIdx.x - seg * lpb);
    const bool active = line < J.nlines;
    const LineOp& op = *J.op;
    const int m = op.m;
    const int L = (m + nseg - 1) / nseg;
    const int s = seg * L;
    const int e = min(s + L, m) - 1;
    const int W = op.kind == 0 ? 40 : 26;
    const long long ies = J.in_es, oes = J.out_es;
    const double* __restrict__ in =
        (J.in_state ? U + (size_t)J.in : J.in) + (long long)line * J.in_ls;
    double* __restrict__ out = J.out + (long long)line * J.out_ls;
    double* __restrict__ tmp = J.tmp + (long long)line * J.out_ls;
    const int base = op.dir == 0 ? -2 : -1;
    const double* __restrict__ lower = op.lower;
    const double* __restrict__ minv = op.minv;
    const double* __restrict__ cpr = op.cprime;
    const int fi = op.first_interior, li = op.last_interior;
    if (active && s <= e) {
        const int fs = max(0, s - W);
        double d = 0.0;
        int r = fs;
        // left closure rows
        for (; r <= e && r < fi; ++r) {
            d = (closure_rhs(op, in, ies, r, J.wall_value) - lower[r] * d) * minv[r];
            if (r >= s) tmp[(long long)r * oes] = d;
        }
        // interior rows: a sliding window of the four inputs, one new load per row, weights
        // already divided by the pivot
        const int ie = min(e, li);
        if (r <= ie) {
            const double* p = in + (long long)(r + base) * ies;
            double p0 = p[0], p1 = p[ies], p2 = p[2 * ies];
            p += 3 * ies;
            const double* __restrict__ wa = op.wa;
            const double* __restrict__ wb = op.wb;
            const double* __restrict__ lm = op.lm;
            if (op.kind == 0) {
#pragma unroll 4
                for (; r <= ie; ++r) {
                    const double p3 = *p;
                    p += ies;
                    d = fma(-lm[r], d, fma(wa[r], p1 + p2, wb[r] * (p0 + p3)));
                    if (r >= s) tmp[(long long)r * oes] = d;
                    p0 = p1;
                    p1 = p2;
                    p2 = p3;
                }
            } else {
#pragma unroll 4
                for (; r <= ie; ++r) {
                    const double p3 = *p;
                    p += ies;
                    d = fma(-lm[r], d, fma(wa[r], p2 - p1, wb[r] * (p3 - p0)));
                    if (r >= s) tmp[(long long)r * oes] = d;
                    p0 = p1;
                    p1 = p2;
                    p2 = p3;
                }
            }
        }
        // right closure rows
        for (; r <= e; ++r) {
            d = (closure_rhs(op, in, ies, r, J.wall_value) - lower[r] * d) * minv[r];
            if (r >= s) tmp[(long long)r * oes] = d;
        }
    }
    __syncthreads();
    if (active && s <= e) {
        const int be = min(e + W, m - 1);
        const double* __restrict__ met = J.metric;
        const bool neg = J.scale < 0.0;
        double y = tmp[(long long)be * oes];
        if (be <= e) {
            const double v = met ? y * met[be] : y;
            out[(long long)be * oes] = neg ? -v : v;
        }
        int r = be - 1;
        // warm-up rows beyond the segment
        for (; r > e; --r) y = tmp[(long long)r * oes] - cpr[r] * y;
        if (met && neg) {
#pragma unroll 4
            for (; r >= s; --r) {
                y = tmp[(long long)r * oes] - cpr[r] * y;
                out[(long long)r * oes] = -y * met[r];
            }
        } else if (met) {
#pragma unroll 4
            for (; r >= s; --r) {
                y = tmp[(long long)r * oes] - cpr[r] * y;
                out[(long long)r * oes] = y * met[r];
            }
        } else {
#pragma unroll 4
            for (; r >= s; --r) {
                y = tmp[(long long)r * oes] - cpr[r] * y;
                out[(long long)r * oes] = neg ? -y : y;
            }
        }
    }
}

}  // namespace

cudaError_t launch_lines(const LineJob* d_jobs, int njobs, int max_blocks, const double* U,
                         cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    dim3 block(LINE_BLOCK);
    dim3 grid(max_blocks, njobs);
    k_lines<<<grid, block, 0, s>>>(d_jobs, U);
    return cudaGetLastError();
}

}  // namespace hyp
