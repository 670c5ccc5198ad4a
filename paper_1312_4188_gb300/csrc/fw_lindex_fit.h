// Host side of the learned index's locator: the per-segment line fit and its
// exact error bound (plain C++, no device code; the device lookup in
// fw_lindex.cu evaluates the same single-precision steps).
//
// Keys of one field live in [0, 2^bits). B holds the sorted starts of the
// elementary intervals (B[0] = 0); the interval of key v is the last t with
// B[t] <= v. The key space is cut into nseg equal segments (segment s covers
// [s << shift, (s + 1) << shift)); each gets a line pos ~ a * (v - base) + b
// with a >= 0 and the largest |predicted - true interval| over its keys, so the
// window [p - E[s], p + E[s]] around a prediction p always holds the interval.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <vector>

namespace fwk {

// Host twin of the device prediction (identical IEEE single-precision steps).
inline int predict(float a, float b, uint32_t v, uint32_t base, int64_t M) {
    const float pf = std::fmaf(a, static_cast<float>(v - base), b);
    return (int)std::floor(std::fmin(std::fmax(pf, 0.0f), (float)(M - 1)));
}

// Exact maximum error of the line (a, b) over every elementary interval that
// meets the segment [base, end), evaluated at the clipped interval ends (the
// prediction is non-decreasing inside a segment, so the ends bound it).
inline int32_t segment_error(const std::vector<uint32_t> &B, int64_t t0, int64_t t1, uint64_t base, uint64_t end,
                             uint64_t dom_end, float a, float b) {
    const int64_t M = (int64_t)B.size();
    int32_t e = 0;
    for (int64_t t = t0; t <= t1 && t < M; ++t) {
        const uint64_t lo = std::max<uint64_t>(B[t], base);
        const uint64_t hi = std::min<uint64_t>((t + 1 < M ? (uint64_t)B[t + 1] : dom_end) - 1, end - 1);
        if (lo > hi) continue;
        const int p0 = predict(a, b, (uint32_t)lo, (uint32_t)base, M);
        const int p1 = predict(a, b, (uint32_t)hi, (uint32_t)base, M);
        e = std::max<int32_t>(e, (int32_t)std::max<int64_t>(std::llabs(p0 - t), std::llabs(p1 - t)));
    }
    return e;
}

// One line per segment of the key space. Two candidates are fit and the one
// with the smaller exact error bound is kept: the least-squares line over the
// (key - base, position) pairs of the interval ends inside the segment, and
// the chord from the position at the segment's first key to the position at
// its last key (the least-squares line alone can extrapolate badly when the
// ends inside a segment are bunched together).
inline void fit_field(const std::vector<uint32_t> &B, int bits, int nseg, int shift, std::vector<float> &A,
                      std::vector<float> &Bc, std::vector<int32_t> &E, int32_t &max_err) {
    const int64_t M = (int64_t)B.size();
    A.assign(nseg, 0.0f);
    Bc.assign(nseg, 0.0f);
    E.assign(nseg, 0);
    max_err = 0;
    const uint64_t dom_end = uint64_t(1) << bits;
    int64_t j = 0;  // first interval start >= base of the segment
    for (int s = 0; s < nseg; ++s) {
        const uint64_t base = (uint64_t)s << shift, end = std::min<uint64_t>(((uint64_t)(s + 1) << shift), dom_end);
        while (j < M && B[j] < base) ++j;
        int64_t j_end = j;
        while (j_end < M && B[j_end] < end) ++j_end;
        const int64_t t0 = (j < M && B[j] == base) ? j : j - 1;  // interval holding `base`
        const int64_t t1 = j_end - 1 >= t0 ? j_end - 1 : t0;     // interval holding end - 1
        // chord
        const double span = (double)(end - 1 - base);
        float ca = span > 0 ? (float)((double)(t1 - t0) / span) : 0.0f;
        float cb = (float)t0;
        int32_t ce = segment_error(B, t0, t1, base, end, dom_end, ca, cb);
        // least squares over the interval starts inside the segment
        const int64_t cnt = j_end - j;
        float la = 0.0f, lb = (float)t0;
        if (cnt >= 2) {
            double sx = 0, sy = 0, sxx = 0, sxy = 0;
            for (int64_t t = j; t < j_end; ++t) {
                const double x = (double)(B[t] - base), y = (double)t;
                sx += x;
                sy += y;
                sxx += x * x;
                sxy += x * y;
            }
            const double den = cnt * sxx - sx * sx;
            if (den > 0) {
                const double a = std::max(0.0, (cnt * sxy - sx * sy) / den);
                la = (float)a;
                lb = (float)((sy - a * sx) / cnt);
            }
        }
        const int32_t le = segment_error(B, t0, t1, base, end, dom_end, la, lb);
        if (le < ce) {
            ca = la;
            cb = lb;
            ce = le;
        }
        A[s] = ca;
        Bc[s] = cb;
        E[s] = ce;
        max_err = std::max(max_err, ce);
    }
}

}  // namespace fwk
