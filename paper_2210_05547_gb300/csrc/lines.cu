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

__device__ __forceinline__ double row_rhs(const LineOp& op, const double* __restrict__ in,
                                          long long ies, int r, int base, double wall, int& c) {
    if (r >= op.first_interior && r <= op.last_interior) {
        const double* p = in + (long long)(r + base) * ies;
        const double p0 = p[0], p1 = p[ies], p2 = p[2 * ies], p3 = p[3 * ies];
        if (op.kind == 0) return op.wi[1] * (p1 + p2) + op.wi[0] * (p0 + p3);
        return op.wi[2] * (p2 - p1) + op.wi[3] * (p3 - p0);
    }
    while (op.crow[c] != r) ++c;
    double v = op.gw[c] * wall;
    const double* p = in + (long long)op.cstart[c] * ies;
    for (int k = 0; k < op.cnum[c]; ++k) v += op.cw[c][k] * p[(long long)k * ies];
    return v;
}

__global__ void __launch_bounds__(128) k_lines(const LineJob* __restrict__ jobs,
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
    if (active && s <= e) {
        int c = 0;
        const int fs = max(0, s - W);
        double d = 0.0;
        for (int r = fs; r <= e; ++r) {
            const double rhs = row_rhs(op, in, ies, r, base, J.wall_value, c);
            d = (rhs - lower[r] * d) * minv[r];
            if (r >= s) tmp[(long long)r * oes] = d;
        }
    }
    __syncthreads();
    if (active && s <= e) {
        const int be = min(e + W, m - 1);
        const double* __restrict__ met = J.metric;
        const double sc = J.scale;
        double y = tmp[(long long)be * oes];
        if (be <= e) {
            double v = sc * y;
            if (met) v *= met[be];
            out[(long long)be * oes] = v;
        }
        for (int r = be - 1; r >= s; --r) {
            y = tmp[(long long)r * oes] - cpr[r] * y;
            if (r <= e) {
                double v = sc * y;
                if (met) v *= met[r];
                out[(long long)r * oes] = v;
            }
        }
    }
}

}  // namespace

cudaError_t launch_lines(const LineJob* d_jobs, int njobs, int max_blocks, const double* U,
                         cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    dim3 block(128);
    dim3 grid(max_blocks, njobs);
    k_lines<<<grid, block, 0, s>>>(d_jobs, U);
    return cudaGetLastError();
}

}  // namespace hyp
