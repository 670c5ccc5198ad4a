// CPU check of the learned index's locator fit (fw_lindex_fit.h). For every key
// tested -- the first and last key of every elementary interval, of every
// segment, and random keys -- the true interval (the last t with B[t] <= v,
// found by std::upper_bound) lies within the stored error of the prediction, so
// the device's verified window never needs its fallback search.
//
// usage: lindex_fit_check <seed> <bits> <nseg> <intervals> <shape>
//   shape 0: interval starts uniform over the key space
//   shape 1: starts bunched in a few narrow clusters (prefix-like)
//   shape 2: every key an interval start (the densest case; bits <= 16)
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "fw_lindex_fit.h"

int main(int argc, char **argv) {
    if (argc != 6) return 2;
    const uint64_t seed = std::strtoull(argv[1], nullptr, 10);
    const int bits = std::atoi(argv[2]), nseg = std::atoi(argv[3]), shape = std::atoi(argv[5]);
    const int64_t want = std::atoll(argv[4]);
    std::mt19937_64 rng(seed);
    const uint64_t dom_end = uint64_t(1) << bits;
    std::vector<uint64_t> ends{0};
    if (shape == 2) {
        for (uint64_t v = 1; v < dom_end; ++v) ends.push_back(v);
    } else {
        std::uniform_int_distribution<uint64_t> U(0, dom_end - 1);
        std::vector<uint64_t> centres;
        for (int c = 0; c < 6; ++c) centres.push_back(U(rng));
        for (int64_t i = 0; i < want; ++i) {
            uint64_t v = U(rng);
            if (shape == 1) {
                const uint64_t c = centres[(size_t)(rng() % centres.size())];
                const uint64_t w = std::max<uint64_t>(1, dom_end >> 12);
                v = std::min(dom_end - 1, c + rng() % w);
            }
            ends.push_back(v);
        }
    }
    std::sort(ends.begin(), ends.end());
    ends.erase(std::unique(ends.begin(), ends.end()), ends.end());
    const std::vector<uint32_t> B(ends.begin(), ends.end());
    const int64_t M = (int64_t)B.size();
    int lg = 0;
    while ((1 << lg) < nseg) ++lg;
    const int shift = bits - lg;
    std::vector<float> A, Bc;
    std::vector<int32_t> E;
    int32_t max_err = -1;
    fwk::fit_field(B, bits, nseg, shift, A, Bc, E, max_err);
    if ((int)A.size() != nseg || (int)E.size() != nseg) return 3;
    int64_t checked = 0, bad = 0;
    int32_t seen = 0;
    auto check = [&](uint64_t v) {
        const uint64_t s = v >> shift, base = s << shift;
        const int p = fwk::predict(A[s], Bc[s], (uint32_t)v, (uint32_t)base, M);
        const int64_t t = (int64_t)(std::upper_bound(B.begin(), B.end(), (uint32_t)v) - B.begin()) - 1;
        const int64_t d = std::llabs((int64_t)p - t);
        seen = std::max<int32_t>(seen, (int32_t)d);
        ++checked;
        if (A[s] < 0.0f || d > E[s] || E[s] > max_err) {
            if (bad++ < 5)
                std::fprintf(stderr, "key %llu: segment %llu predicted %d, interval %lld, stored error %d\n",
                             (unsigned long long)v, (unsigned long long)s, p, (long long)t, E[s]);
        }
    };
    for (int64_t t = 0; t < M; ++t) {
        check(B[t]);
        check((t + 1 < M ? (uint64_t)B[t + 1] : dom_end) - 1);
    }
    for (int s = 0; s < nseg; ++s) {
        const uint64_t base = (uint64_t)s << shift;
        check(base);
        check(std::min(base + (uint64_t(1) << shift), dom_end) - 1);
    }
    std::uniform_int_distribution<uint64_t> U(0, dom_end - 1);
    for (int i = 0; i < 200000; ++i) check(U(rng));
    std::printf("%lld %lld %d %d %lld\n", (long long)checked, (long long)bad, max_err, seen, (long long)M);
    return bad == 0 ? 0 : 1;
}
