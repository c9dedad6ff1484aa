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
//
// Past the first ~20 interior rows the Thomas factors are bitwise constant (LineOp::rc), so those
// rows take their factors from registers and only the field values come from memory. A thread
// has only a few FP64 instructions per row and the grid holds a few warps per sub-partition, so
// the rows of that constant stretch are software-pipelined: the loads for row r + 8 are issued
// while row r is computed.
//
// Under HYP_MIXED that constant stretch leaves the FP64 pipe. Jobs marked f32ok (the
// interpolations and derivatives that feed only the diffusive fluxes) run it in plain binary32:
// inputs are rounded with integer instructions, the recurrences run on the FP32 pipe, the forward
// values of those rows are kept as binary32 in the first half of their 8-byte storage slot, and
// outputs are widened back to binary64. The other derivatives (those feeding the convective
// fluxes, the pressure and the divergences) form the adjacent differences of their inputs in
// binary64 and run the recurrence in binary32 on those derivative-sized values (fwd_rows_cdiff).
// The other interpolations run it in double-word arithmetic (dword.cuh): each binary64 input is
// split into a pair of binary32 numbers, and the recurrences carry their rounding errors in the
// low word (error-free sums and FMA products, about 48 significand bits). The forward values are
// kept as a binary32 pair in the 8-byte slot, and each output is the binary64 sum of its pair.
// Closure rows and the first interior rows stay FP64.
#include "dword.cuh"
#include "fp32.cuh"
#include "internal.h"

namespace hyp {
namespace {

constexpr int PF = 8;   // prefetch distance (rows) of the constant-factor loops
// the same for the double-word rows (16 or 24 rows were measured slower: the registers cost more
// resident warps than the earlier loads gain)
constexpr int PF_DW = 8;

__device__ __forceinline__ double closure_rhs(const LineOp& op, const double* __restrict__ in,
                                              long long ies, int r, double wall) {
    int c = 0;
    while (op.crow[c] != r) ++c;
    double v = op.gw[c] * wall;
    const double* p = in + (long long)op.cstart[c] * ies;
    for (int k = 0; k < op.cnum[c]; ++k) v += op.cw[c][k] * p[(long long)k * ies];
    return v;
}

// Sliding window of the four inputs of an interior row: p0..p2 held, p3 the new one.
struct Window {
    double p0, p1, p2;
};

template <int KIND>
__device__ __forceinline__ double interior_row(double d, const Window& w, double p3, double wa,
                                               double wb, double lm) {
    if (KIND == 0) return fma(-lm, d, fma(wa, w.p1 + w.p2, wb * (w.p0 + p3)));
    return fma(-lm, d, fma(wa, w.p2 - w.p1, wb * (p3 - w.p0)));
}

__device__ __forceinline__ void shift(Window& w, double p3) {
    w.p0 = w.p1;
    w.p1 = w.p2;
    w.p2 = p3;
}

// Interior rows r..r1 with per-row factors; `p` points at the new input of row r and is advanced
// past row r1.
template <int KIND, bool STORE>
__device__ __forceinline__ void fwd_rows_var(int r, int r1, double& d, Window& w,
                                             const double* __restrict__& p, long long ies,
                                             const LineOp& op, double* __restrict__ tmp,
                                             long long oes) {
    const double* __restrict__ wa = op.wa;
    const double* __restrict__ wb = op.wb;
    const double* __restrict__ lm = op.lm;
#pragma unroll 2
    for (; r <= r1; ++r) {
        const double p3 = *p;
        p += ies;
        d = interior_row<KIND>(d, w, p3, wa[r], wb[r], lm[r]);
        if (STORE) tmp[(long long)r * oes] = d;
        shift(w, p3);
    }
}

// Interior rows r..r1 with the constant factors, inputs prefetched PF rows ahead.
template <int KIND, bool STORE>
__device__ __forceinline__ void fwd_rows_const(int r, int r1, double& d, Window& w,
                                               const double* __restrict__& p, long long ies,
                                               const LineOp& op, double* __restrict__ tmp,
                                               long long oes) {
    const int n = r1 - r + 1;
    if (n <= 0) return;
    const double wa = op.wac, wb = op.wbc, lm = op.lmc;
    const double* __restrict__ pp = p;
    double q[PF];
#pragma unroll
    for (int k = 0; k < PF; ++k) q[k] = k < n ? pp[(long long)k * ies] : 0.0;
    for (; r + PF - 1 <= r1; r += PF) {
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            const double p3 = q[k];
            q[k] = r + PF + k <= r1 ? pp[(long long)(PF + k) * ies] : 0.0;
            d = interior_row<KIND>(d, w, p3, wa, wb, lm);
            if (STORE) tmp[(long long)(r + k) * oes] = d;
            shift(w, p3);
        }
        pp += PF * ies;
    }
#pragma unroll
    for (int k = 0; k < PF - 1; ++k) {
        if (r + k <= r1) {
            const double p3 = q[k];
            d = interior_row<KIND>(d, w, p3, wa, wb, lm);
            if (STORE) tmp[(long long)(r + k) * oes] = d;
            shift(w, p3);
        }
    }
    p += (long long)n * ies;
}

__device__ __forceinline__ float* slot32(double* p) { return reinterpret_cast<float*>(p); }
__device__ __forceinline__ const float* slot32(const double* p) {
    return reinterpret_cast<const float*>(p);
}

template <int KIND>
__device__ __forceinline__ float interior_row32(float d, float p0, float p1, float p2, float p3,
                                                float wa, float wb, float lm) {
    if (KIND == 0) return fmaf(-lm, d, fmaf(wa, p1 + p2, wb * (p0 + p3)));
    return fmaf(-lm, d, fmaf(wa, p2 - p1, wb * (p3 - p0)));
}

// The constant-factor rows r..r1 in binary32 (f32ok jobs under HYP_MIXED).
template <int KIND, bool STORE>
__device__ __forceinline__ void fwd_rows_const32(int r, int r1, double& d, Window& w,
                                                 const double* __restrict__& p, long long ies,
                                                 const LineOp& op, double* __restrict__ tmp,
                                                 long long oes) {
    const int n = r1 - r + 1;
    if (n <= 0) return;
    const float wa = op.wac_f, wb = op.wbc_f, lm = op.lmc_f;
    const double* __restrict__ pp = p;
    float df = f32_of(d), p0 = f32_of(w.p0), p1 = f32_of(w.p1), p2 = f32_of(w.p2);
    double q[PF];   // raw prefetched inputs; rounded when used so the load latency stays hidden
#pragma unroll
    for (int k = 0; k < PF; ++k) q[k] = k < n ? pp[(long long)k * ies] : 0.0;
    for (; r + PF - 1 <= r1; r += PF) {
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            const float p3 = f32_of(q[k]);
            q[k] = r + PF + k <= r1 ? pp[(long long)(PF + k) * ies] : 0.0;
            df = interior_row32<KIND>(df, p0, p1, p2, p3, wa, wb, lm);
            if (STORE) *slot32(tmp + (long long)(r + k) * oes) = df;
            p0 = p1;
            p1 = p2;
            p2 = p3;
        }
        pp += PF * ies;
    }
#pragma unroll
    for (int k = 0; k < PF - 1; ++k) {
        if (r + k <= r1) {
            const float p3 = f32_of(q[k]);
            df = interior_row32<KIND>(df, p0, p1, p2, p3, wa, wb, lm);
            if (STORE) *slot32(tmp + (long long)(r + k) * oes) = df;
            p0 = p1;
            p1 = p2;
            p2 = p3;
        }
    }
    d = f64_of(df);
    w.p0 = f64_of(p0);
    w.p1 = f64_of(p1);
    w.p2 = f64_of(p2);
    p += (long long)n * ies;
}

// The row's right-hand side is formed off the recurrence's dependency chain; the recurrence step
// itself is dw_step (one binary32 product and sum on the chain of the high word).
template <int KIND>
__device__ __forceinline__ dword interior_row_dw(dword d, dword p0, dword p1, dword p2, dword p3,
                                                 dword wa, dword wb, dword lm) {
    const dword s1 = KIND == 0 ? dw_add(p1, p2) : dw_sub(p2, p1);
    const dword s2 = KIND == 0 ? dw_add(p0, p3) : dw_sub(p3, p0);
    return dw_step(d, dw_add(dw_mul(wa, s1), dw_mul(wb, s2)), lm);
}

// The constant-factor rows r..r1 in double-word arithmetic (jobs not marked f32ok under
// HYP_MIXED). The window keeps each input both as binary64 (handed back to the FP64 rows that
// follow) and as a double word.
template <int KIND, bool STORE>
__device__ __forceinline__ void fwd_rows_constdw(int r, int r1, double& d, Window& w,
                                                 const double* __restrict__& p, long long ies,
                                                 const LineOp& op, double* __restrict__ tmp,
                                                 long long oes) {
    const int n = r1 - r + 1;
    if (n <= 0) return;
    const dword wa{op.wac_f, op.wac_l}, wb{op.wbc_f, op.wbc_l}, lm{op.lmc_f, op.lmc_l};
    const double* __restrict__ pp = p;
    dword dd = dw_of(d), p0 = dw_of(w.p0), p1 = dw_of(w.p1), p2 = dw_of(w.p2);
    double q[PF_DW];
#pragma unroll
    for (int k = 0; k < PF_DW; ++k) q[k] = k < n ? pp[(long long)k * ies] : 0.0;
    for (; r + PF_DW - 1 <= r1; r += PF_DW) {
#pragma unroll
        for (int k = 0; k < PF_DW; ++k) {
            const double x3 = q[k];
            const dword p3 = dw_of(x3);
            q[k] = r + PF_DW + k <= r1 ? pp[(long long)(PF_DW + k) * ies] : 0.0;
            dd = interior_row_dw<KIND>(dd, p0, p1, p2, p3, wa, wb, lm);
            if (STORE) dw_store(tmp + (long long)(r + k) * oes, dd);
            p0 = p1;
            p1 = p2;
            p2 = p3;
            shift(w, x3);
        }
        pp += PF_DW * ies;
    }
#pragma unroll
    for (int k = 0; k < PF_DW - 1; ++k) {
        if (r + k <= r1) {
            const double x3 = q[k];
            const dword p3 = dw_of(x3);
            dd = interior_row_dw<KIND>(dd, p0, p1, p2, p3, wa, wb, lm);
            if (STORE) dw_store(tmp + (long long)(r + k) * oes, dd);
            p0 = p1;
            p1 = p2;
            p2 = p3;
            shift(w, x3);
        }
    }
    d = dw_to_f64(dd);
    p += (long long)n * ies;
}

// The constant-factor rows r..r1 of a derivative (KIND 1) under HYP_MIXED, jobs not marked
// f32ok. The row's right-hand side wa (p2 - p1) + wb (p3 - p0) is built from the adjacent
// differences of the inputs: each difference is formed in binary64 and rounded to binary32. A
// difference of neighbours within a factor of two is exact in binary64, else within an ulp of
// itself. p3 - p0 is the sum of three adjacent differences. The recurrence then runs in binary32
// on derivative-sized values. Their rounding is relative to the derivative, not to the field it
// differentiates: the cancellation that made binary32 inputs miss the error bound happens in
// the binary64 differences.
template <bool STORE>
__device__ __forceinline__ void fwd_rows_cdiff(int r, int r1, double& d, Window& w,
                                               const double* __restrict__& p, long long ies,
                                               const LineOp& op, double* __restrict__ tmp,
                                               long long oes) {
    const int n = r1 - r + 1;
    if (n <= 0) return;
    const float wa = op.wac_f, wb = op.wbc_f, lm = op.lmc_f;
    const double* __restrict__ pp = p;
    float df = f32_of(d);
    float e1 = f32_of(w.p1 - w.p0), e2 = f32_of(w.p2 - w.p1);
    double q[PF];
#pragma unroll
    for (int k = 0; k < PF; ++k) q[k] = k < n ? pp[(long long)k * ies] : 0.0;
    for (; r + PF - 1 <= r1; r += PF) {
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            const double x3 = q[k];
            q[k] = r + PF + k <= r1 ? pp[(long long)(PF + k) * ies] : 0.0;
            const float e3 = f32_of(x3 - w.p2);
            const float rhs = fmaf(wa, e2, __fmul_rn(wb, __fadd_rn(__fadd_rn(e1, e2), e3)));
            df = fmaf(-lm, df, rhs);
            if (STORE) *slot32(tmp + (long long)(r + k) * oes) = df;
            e1 = e2;
            e2 = e3;
            shift(w, x3);
        }
        pp += PF * ies;
    }
#pragma unroll
    for (int k = 0; k < PF - 1; ++k) {
        if (r + k <= r1) {
            const double x3 = q[k];
            const float e3 = f32_of(x3 - w.p2);
            const float rhs = fmaf(wa, e2, __fmul_rn(wb, __fadd_rn(__fadd_rn(e1, e2), e3)));
            df = fmaf(-lm, df, rhs);
            if (STORE) *slot32(tmp + (long long)(r + k) * oes) = df;
            e1 = e2;
            e2 = e3;
            shift(w, x3);
        }
    }
    d = f64_of(df);
    p += (long long)n * ies;
}

// Forward sweep over rows r..r1 of one kind of region (closure / per-row / constant interior).
template <int KIND, bool STORE, int MODE>
__device__ __forceinline__ void fwd_span(int r, int r1, double& d, Window& w,
                                         const double* __restrict__ in,
                                         const double* __restrict__& p, long long ies,
                                         const LineOp& op, double wall, double* __restrict__ tmp,
                                         long long oes) {
    if (r > r1) return;
    const int fi = op.first_interior, li = op.last_interior, rc = op.rc;
    const int base = op.dir == 0 ? -2 : -1;
    // left closure rows
    for (; r <= r1 && r < fi; ++r) {
        d = (closure_rhs(op, in, ies, r, wall) - op.lower[r] * d) * op.minv[r];
        if (STORE) tmp[(long long)r * oes] = d;
    }
    if (r > r1) return;
    if (r <= li) {
        // (re)load the window when entering the interior here
        if (p == nullptr) {
            const double* q = in + (long long)(r + base) * ies;
            w.p0 = q[0];
            w.p1 = q[ies];
            w.p2 = q[2 * ies];
            p = q + 3 * ies;
        }
        const int rv = min(r1, min(li, rc - 1));
        if (r <= rv) {
            fwd_rows_var<KIND, STORE>(r, rv, d, w, p, ies, op, tmp, oes);
            r = rv + 1;
        }
        const int rcn = min(r1, li);
        if (r <= rcn) {
            if constexpr (MODE == 1) fwd_rows_const32<KIND, STORE>(r, rcn, d, w, p, ies, op, tmp, oes);
            else if constexpr (MODE == 2) fwd_rows_constdw<KIND, STORE>(r, rcn, d, w, p, ies, op, tmp, oes);
            else if constexpr (MODE == 3) fwd_rows_cdiff<STORE>(r, rcn, d, w, p, ies, op, tmp, oes);
            else fwd_rows_const<KIND, STORE>(r, rcn, d, w, p, ies, op, tmp, oes);
            r = rcn + 1;
        }
    }
    // right closure rows
    for (; r <= r1; ++r) {
        d = (closure_rhs(op, in, ies, r, wall) - op.lower[r] * d) * op.minv[r];
        if (STORE) tmp[(long long)r * oes] = d;
    }
}

// Output modes of the back substitution: 0 none (warm-up rows), 1 y, 2 -y, 3 y met, 4 -y met.
template <int OM>
__device__ __forceinline__ void put(double* __restrict__ out, long long oes, int r, double y,
                                    double m) {
    if (OM == 1) out[(long long)r * oes] = y;
    if (OM == 2) out[(long long)r * oes] = -y;
    if (OM == 3) out[(long long)r * oes] = y * m;
    if (OM == 4) out[(long long)r * oes] = -y * m;
}

// Back substitution over rows r0 >= r >= r1 (descending) with per-row c'.
template <int OM>
__device__ __forceinline__ void back_rows_var(int r0, int r1, double& y,
                                              const double* __restrict__ tmp, long long oes,
                                              const double* __restrict__ cpr,
                                              const double* __restrict__ met,
                                              double* __restrict__ out) {
#pragma unroll 2
    for (int r = r0; r >= r1; --r) {
        y = tmp[(long long)r * oes] - cpr[r] * y;
        put<OM>(out, oes, r, y, OM >= 3 ? met[r] : 0.0);
    }
}

// Back substitution over rows r0 >= r >= r1 with the constant c', loads prefetched PF rows ahead.
template <int OM>
__device__ __forceinline__ void back_rows_const(int r0, int r1, double& y,
                                                const double* __restrict__ tmp, long long oes,
                                                double cc, const double* __restrict__ met,
                                                double* __restrict__ out) {
    const int n = r0 - r1 + 1;
    if (n <= 0) return;
    double q[PF], mq[PF];
#pragma unroll
    for (int k = 0; k < PF; ++k) {
        q[k] = k < n ? tmp[(long long)(r0 - k) * oes] : 0.0;
        mq[k] = (OM >= 3 && k < n) ? met[r0 - k] : 0.0;
    }
    int r = r0;
    for (; r - PF + 1 >= r1; r -= PF) {
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            const double t = q[k], m = mq[k];
            const int rn = r - PF - k;
            q[k] = rn >= r1 ? tmp[(long long)rn * oes] : 0.0;
            if (OM >= 3) mq[k] = rn >= r1 ? met[rn] : 0.0;
            y = fma(-cc, y, t);
            put<OM>(out, oes, r - k, y, m);
        }
    }
#pragma unroll
    for (int k = 0; k < PF - 1; ++k) {
        if (r - k >= r1) {
            y = fma(-cc, y, q[k]);
            put<OM>(out, oes, r - k, y, mq[k]);
        }
    }
}

template <int OM>
__device__ __forceinline__ void put32(double* __restrict__ out, long long oes, int r, float y,
                                      float m) {
    if (OM == 1) out[(long long)r * oes] = f64_of(y);
    if (OM == 2) out[(long long)r * oes] = f64_of(-y);
    if (OM == 3) out[(long long)r * oes] = f64_of(y * m);
    if (OM == 4) out[(long long)r * oes] = f64_of(-y * m);
}

// The constant-factor rows r0 >= r >= r1 in binary32, reading the binary32 forward values.
template <int OM>
__device__ __forceinline__ void back_rows_const32(int r0, int r1, double& y,
                                                  const double* __restrict__ tmp, long long oes,
                                                  float cc, const float* __restrict__ met,
                                                  double* __restrict__ out) {
    const int n = r0 - r1 + 1;
    if (n <= 0) return;
    float yf = f32_of(y);
    float q[PF], mq[PF];
#pragma unroll
    for (int k = 0; k < PF; ++k) {
        q[k] = k < n ? *slot32(tmp + (long long)(r0 - k) * oes) : 0.0f;
        mq[k] = (OM >= 3 && k < n) ? met[r0 - k] : 0.0f;
    }
    int r = r0;
    for (; r - PF + 1 >= r1; r -= PF) {
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            const float t = q[k], m = mq[k];
            const int rn = r - PF - k;
            q[k] = rn >= r1 ? *slot32(tmp + (long long)rn * oes) : 0.0f;
            if (OM >= 3) mq[k] = rn >= r1 ? met[rn] : 0.0f;
            yf = fmaf(-cc, yf, t);
            put32<OM>(out, oes, r - k, yf, m);
        }
    }
#pragma unroll
    for (int k = 0; k < PF - 1; ++k) {
        if (r - k >= r1) {
            yf = fmaf(-cc, yf, q[k]);
            put32<OM>(out, oes, r - k, yf, mq[k]);
        }
    }
    y = f64_of(yf);
}

// The constant-factor rows r0 >= r >= r1 in double-word arithmetic, reading the double-word
// forward values; each output is the binary64 sum of its pair (times the metric in binary64).
template <int OM>
__device__ __forceinline__ void back_rows_constdw(int r0, int r1, double& y,
                                                  const double* __restrict__ tmp, long long oes,
                                                  dword cc, const double* __restrict__ met,
                                                  double* __restrict__ out) {
    const int n = r0 - r1 + 1;
    if (n <= 0) return;
    dword yd = dw_of(y);
    dword q[PF_DW];
    double mq[PF_DW];
#pragma unroll
    for (int k = 0; k < PF_DW; ++k) {
        q[k] = k < n ? dw_load(tmp + (long long)(r0 - k) * oes) : dword{0.0f, 0.0f};
        mq[k] = (OM >= 3 && k < n) ? met[r0 - k] : 0.0;
    }
    int r = r0;
    for (; r - PF_DW + 1 >= r1; r -= PF_DW) {
#pragma unroll
        for (int k = 0; k < PF_DW; ++k) {
            const dword t = q[k];
            const double m = mq[k];
            const int rn = r - PF_DW - k;
            q[k] = rn >= r1 ? dw_load(tmp + (long long)rn * oes) : dword{0.0f, 0.0f};
            if (OM >= 3) mq[k] = rn >= r1 ? met[rn] : 0.0;
            yd = dw_step(yd, t, cc);
            if (OM != 0) put<OM>(out, oes, r - k, dw_to_f64(yd), m);
        }
    }
#pragma unroll
    for (int k = 0; k < PF_DW - 1; ++k) {
        if (r - k >= r1) {
            yd = dw_step(yd, q[k], cc);
            if (OM != 0) put<OM>(out, oes, r - k, dw_to_f64(yd), mq[k]);
        }
    }
    y = dw_to_f64(yd);
}

// Back substitution over rows r0 >= r >= r1, split at the constant-factor stretch.
template <int OM, int MODE>
__device__ __forceinline__ void back_span(int r0, int r1, double& y, const LineOp& op,
                                          const double* __restrict__ tmp, long long oes,
                                          const double* __restrict__ met,
                                          const float* __restrict__ met_f,
                                          double* __restrict__ out) {
    if (r0 < r1) return;
    const int li = op.last_interior, rc = op.rc;
    const int a = max(r1, li + 1);            // rows above the interior (right closure)
    if (r0 >= a) back_rows_var<OM>(r0, a, y, tmp, oes, op.cprime, met, out);
    const int c0 = min(r0, li), c1 = max(r1, rc);
    if (c0 >= c1) {
        if (MODE == 1 || MODE == 3) back_rows_const32<OM>(c0, c1, y, tmp, oes, op.cpc_f, met_f, out);
        else if (MODE == 2)
            back_rows_constdw<OM>(c0, c1, y, tmp, oes, dword{op.cpc_f, op.cpc_l}, met, out);
        else back_rows_const<OM>(c0, c1, y, tmp, oes, op.cpc, met, out);
    }
    const int v0 = min(r0, rc - 1);
    if (v0 >= r1) back_rows_var<OM>(v0, r1, y, tmp, oes, op.cprime, met, out);
}

template <int KIND, int MODE>
__device__ __forceinline__ void forward(const LineJob& J, const LineOp& op,
                                        const double* __restrict__ in, double* __restrict__ tmp,
                                        int s, int e, int W, double wall) {
    const int fs = max(0, s - W);
    const long long ies = J.in_es, oes = J.out_es;
    double d = 0.0;
    Window w{0.0, 0.0, 0.0};
    const double* __restrict__ p = nullptr;
    fwd_span<KIND, false, MODE>(fs, s - 1, d, w, in, p, ies, op, wall, tmp, oes);
    fwd_span<KIND, true, MODE>(s, e, d, w, in, p, ies, op, wall, tmp, oes);
}

template <int OM, int MODE>
__device__ __forceinline__ void backward(const LineOp& op, const double* __restrict__ tmp,
                                         long long oes, const double* __restrict__ met,
                                         const float* __restrict__ met_f,
                                         double* __restrict__ out, int s, int e, int be) {
    // the last row is a closure row (FP64 storage) or, for lines without one, an interior row
    const bool last_c = MODE != 0 && be >= op.rc && be <= op.last_interior;
    double y;
    if (last_c && (MODE == 1 || MODE == 3)) y = f64_of(*slot32(tmp + (long long)be * oes));
    else if (last_c) y = dw_to_f64(dw_load(tmp + (long long)be * oes));
    else y = tmp[(long long)be * oes];
    if (be <= e) put<OM>(out, oes, be, y, OM >= 3 ? met[be] : 0.0);
    back_span<0, MODE>(be - 1, e + 1, y, op, tmp, oes, met, met_f, out);   // warm-up rows
    back_span<OM, MODE>(min(be - 1, e), s, y, op, tmp, oes, met, met_f, out);
}

template <int MODE>
__device__ __forceinline__ void run_line(const LineJob& J, const LineOp& op,
                                         const double* __restrict__ in, double* __restrict__ out,
                                         double* __restrict__ tmp, int s, int e, int m, int W,
                                         bool active, double wall) {
    if (active && s <= e) {
        if constexpr (MODE == 3) forward<1, MODE>(J, op, in, tmp, s, e, W, wall);   // derivatives only
        else if (op.kind == 0) forward<0, MODE>(J, op, in, tmp, s, e, W, wall);
        else forward<1, MODE>(J, op, in, tmp, s, e, W, wall);
    }
    __syncthreads();
    if (active && s <= e) {
        const int be = min(e + W, m - 1);
        const double* __restrict__ met = J.metric;
        const float* __restrict__ met_f = J.metric_f;
        const bool neg = J.scale < 0.0;
        const long long oes = J.out_es;
        if (met) {
            if (neg) backward<4, MODE>(op, tmp, oes, met, met_f, out, s, e, be);
            else backward<3, MODE>(op, tmp, oes, met, met_f, out, s, e, be);
        } else {
            if (neg) backward<2, MODE>(op, tmp, oes, met, met_f, out, s, e, be);
            else backward<1, MODE>(op, tmp, oes, met, met_f, out, s, e, be);
        }
    }
}

// One instantiation per precision: the FP64 one carries only the binary64 sweeps (and keeps its
// registers), the HYP_MIXED one the binary32 and double-word sweeps beside the binary64 rows.
template <bool MIXED>
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
    long long ioff, ooff;
    if (J.lpp) {
        const int k = line / J.lpp, l = line - k * J.lpp;
        ioff = k * J.in_ps + (long long)l * J.in_ls;
        ooff = k * J.out_ps + (long long)l * J.out_ls;
    } else {
        ioff = (long long)line * J.in_ls;
        ooff = (long long)line * J.out_ls;
    }
    const double* __restrict__ in = (J.in_state ? U + (size_t)J.in : J.in) + ioff;
    double* __restrict__ out = J.out + ooff;
    double* __restrict__ tmp = J.tmp + ooff;
    const double wall = (J.wall_arr && active) ? J.wall_arr[line] : J.wall_value;
    // uniform per block: every thread of a block works on the same job
    if constexpr (MIXED) {
        if (J.f32ok) run_line<1>(J, op, in, out, tmp, s, e, m, W, active, wall);
        else if (op.kind == 1) run_line<3>(J, op, in, out, tmp, s, e, m, W, active, wall);
        else run_line<2>(J, op, in, out, tmp, s, e, m, W, active, wall);
    } else {
        run_line<0>(J, op, in, out, tmp, s, e, m, W, active, wall);
    }
}

}  // namespace

cudaError_t launch_lines(const LineJob* d_jobs, int njobs, int max_blocks, const double* U,
                         cudaStream_t s, int mixed) {
    if (njobs == 0) return cudaSuccess;
    dim3 block(LINE_BLOCK);
    dim3 grid(max_blocks, njobs);
    if (mixed) k_lines<true><<<grid, block, 0, s>>>(d_jobs, U);
    else k_lines<false><<<grid, block, 0, s>>>(d_jobs, U);
    return cudaGetLastError();
}

}  // namespace hyp
