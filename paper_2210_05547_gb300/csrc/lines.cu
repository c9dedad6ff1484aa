// Batched compact staggered line operators (Sec. 3.1): y = A^{-1} B x along grid lines.
//
// One thread owns one grid line of one job. Lines along y (stride = row pitch) are read with
// adjacent threads on adjacent columns, so every step is a coalesced row access. Lines along x
// walk contiguous memory per thread; a warp then touches 32 rows per step and relies on L1 to
// serve the next 15 steps from the same 128-byte sectors.
#include "internal.h"

namespace hyp {
namespace {

__global__ void __launch_bounds__(128) k_lines(const LineJob* __restrict__ jobs,
                                               const double* __restrict__ U) {
    const LineJob& J = jobs[blockIdx.y];
    const int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= J.nlines) return;
    const LineOp& op = *J.op;
    const double* __restrict__ in =
        (J.in_state ? U + (size_t)J.in : J.in) + line * J.in_ls;
    double* __restrict__ out = J.out + line * J.out_ls;
    double* __restrict__ tmp = (J.tmp ? J.tmp : J.out) + line * J.out_ls;
    const long long ies = J.in_es, oes = J.out_es;
    const int m = op.m;
    // interior input offset: face output r reads centres r-2..r+1; centre output r reads faces r-1..r+2
    const int base = op.dir == 0 ? -2 : -1;
    const double w0 = op.wi[0], w1 = op.wi[1], w2 = op.wi[2], w3 = op.wi[3];
    double dprev = 0.0;
    int c = 0;   // next closure row
    for (int r = 0; r < m; ++r) {
        double rhs;
        if (r >= op.first_interior && r <= op.last_interior) {
            const double* p = in + (r + base) * ies;
            rhs = w0 * p[0] + w1 * p[ies] + w2 * p[2 * ies] + w3 * p[3 * ies];
        } else {
            while (op.crow[c] != r) ++c;
            rhs = op.gw[c] * J.wall_value;
            const double* p = in + op.cstart[c] * ies;
            for (int k = 0; k < op.cnum[c]; ++k) rhs += op.cw[c][k] * p[k * ies];
        }
        const double d = (rhs - op.lower[r] * dprev) * op.minv[r];
        tmp[r * oes] = d;
        dprev = d;
    }
    const double* __restrict__ met = J.metric;
    const double sc = J.scale;
    double y = dprev;
    for (int r = m - 1; r >= 0; --r) {
        if (r < m - 1) y = tmp[r * oes] - op.cprime[r] * y;
        double v = sc * y;
        if (met) v *= met[r];
        if (J.accumulate) v += out[r * oes];
        out[r * oes] = v;
    }
}

}  // namespace

cudaError_t launch_lines(const LineJob* d_jobs, int njobs, int max_lines, const double* U,
                         cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    dim3 block(128);
    dim3 grid((max_lines + 127) / 128, njobs);
    k_lines<<<grid, block, 0, s>>>(d_jobs, U);
    return cudaGetLastError();
}

}  // namespace hyp
