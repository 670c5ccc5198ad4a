// Bucket filter: the per-packet first-match routine shared by the packet-split
// filter kernel (fw_filter.cu) and the batched persistent kernel (fw_batch.cu).
//
// A rule set whose partition class sub-lists hold at most kFilterMaxRecords
// records carries a filter block (layout: filter_layout in fw_internal.cuh):
//  - per class c and bucket table t, 256 rows of W 32-bit words, bit j of a row
//    set when record j of c's sub-list can hold a packet of that bucket:
//      t = 0: top 8 bits of the source address,
//      t = 1: top 8 bits of the destination address,
//      t = 2: (sport >> 12) << 4 | (dport >> 12);
//  - per class {first stored record, exact mask words 0 and 1, 0}, and the
//    exact mask of every word (bit j set when record j's fields are unions of
//    whole buckets, so that its bits alone decide it);
//  - per record an exact-test record (two uint4) and a verdict word
//    (original rule index | action << 31);
//  - the protocol -> protocol class table;
//  - for rows wider than two words, a summary of each row (bit w set when
//    word w is not zero).
// A rule that contains the packet has its bit set in all three of the
// packet's rows (each of its field sets holds the packet's value, so it meets
// that value's bucket): the AND of the rows is a superset of the matching
// records. Candidates are tested in increasing record order, and the first that
// passes is the packet's first match in its class sub-list, i.e. in the list.
#pragma once

#include "fw_scan.cuh"

namespace fwk {

// What a kernel needs to read a filter block: 32-bit byte offsets of its parts,
// the partition's class count and address key, and the row width.
struct FilterView {
    int32_t tables, classes, exact, recs, verdicts, class_of;
    int32_t n_classes, key_field, key_bits, words;
};

inline FilterView filter_view(const fw_ruleset *rs) {
    const int64_t records = rs->class_off[kMaxClasses - 1] + rs->class_len[kMaxClasses - 1];
    const FilterLayout L = filter_layout(rs->n_classes, rs->filter_words, records);
    FilterView v;
    v.tables = (int32_t)L.tables;
    v.classes = (int32_t)L.classes;
    v.exact = (int32_t)L.exact;
    v.recs = (int32_t)L.recs;
    v.verdicts = (int32_t)L.verdicts;
    v.class_of = (int32_t)L.class_of;
    v.n_classes = rs->n_classes;
    v.key_field = rs->key_bits == 0 ? 0 : rs->key_field;
    v.key_bits = rs->key_bits;
    v.words = rs->filter_words;
    return v;
}

// Non-zero exactly when the packet is outside the record's rule. The record is
// {saddr & smask, smask, daddr & dmask, dmask} and {-sport_lo, sport_hi -
// sport_lo, -dport_lo, dport_hi - dport_lo} (mod 2^32): two 3-input logic ops
// for the addresses, a multiply-add (`one` = 1 at run time, so it is issued on
// the FMA pipe) and an unsigned compare per port, chained into one predicate.
__device__ __forceinline__ uint32_t filter_mismatch(uint32_t s, uint32_t d, uint32_t sp, uint32_t dp, const uint4 &a,
                                                    const uint4 &b, uint32_t one) {
    const uint32_t ts = sp * one + b.x;
    const uint32_t td = dp * one + b.z;
    uint32_t r;
    asm("{\n\t"
        ".reg .pred q;\n\t"
        ".reg .b32 t;\n\t"
        "setp.gt.u32 q, %1, %2;\n\t"
        "lop3.or.b32 t|q, %3, %4, %5, 0x28, q;\n\t"
        "lop3.or.b32 t|q, %6, %7, %8, 0x28, q;\n\t"
        "setp.gt.or.u32 q, %9, %10, q;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t"
        "}"
        : "=r"(r)
        : "r"(ts), "r"(b.y), "r"(s), "r"(a.x), "r"(a.y), "r"(d), "r"(a.z), "r"(a.w), "r"(td), "r"(b.w));
    return r;
}

// The packet's partition class (KEY: 0 no address key, 1 source, 2 destination, -1 read from v).
template <int KEY>
__device__ __forceinline__ uint32_t filter_class(const unsigned char *base, const FilterView &v, uint32_t s,
                                                 uint32_t d, uint32_t pr) {
    uint32_t c = base[v.class_of + pr];
    const int key = KEY >= 0 ? KEY : v.key_field;
    if (key != 0) c = (c << v.key_bits) | ((key == 1 ? s : d) >> (32 - v.key_bits));
    return c;
}

template <int W>
using FilterMask = typename std::conditional<W == 1, uint32_t, uint64_t>::type;

// Rows of one or two words (W = 1, 2): the three rows' AND as one integer.
template <int W, int KEY>
__device__ __forceinline__ FilterMask<W> filter_candidates(const unsigned char *base, const FilterView &v,
                                                           uint32_t s, uint32_t d, uint32_t sp, uint32_t dp,
                                                           uint32_t pr, uint32_t &cls) {
    using M = FilterMask<W>;
    const uint32_t c = filter_class<KEY>(base, v, s, d, pr);
    cls = c;
    const M *T = reinterpret_cast<const M *>(base + v.tables) + c * 768u;
    return T[s >> 24] & T[256u + (d >> 24)] & T[512u + (((sp >> 12) << 4) | (dp >> 12))];
}

// First candidate of m (W = 1, 2) that passes its exact test: its verdict word, or ~0u.
template <int W>
__device__ __forceinline__ uint32_t filter_first(const unsigned char *base, const FilterView &v, FilterMask<W> m,
                                                 uint32_t cls, uint32_t s, uint32_t d, uint32_t sp, uint32_t dp,
                                                 uint32_t one) {
    using M = FilterMask<W>;
    if (m == 0) return 0xFFFFFFFFu;
    // class info: first stored record, exact mask (low, high word); one-word rows read only the
    // first eight bytes (half the shared-memory wavefronts of the 16-byte entry)
    uint32_t first;
    M ex;
    if constexpr (W == 1) {
        const uint2 ci = reinterpret_cast<const uint2 *>(base + v.classes)[2 * cls];
        first = ci.x;
        ex = (M)ci.y;
    } else {
        const uint4 ci = reinterpret_cast<const uint4 *>(base + v.classes)[cls];
        first = ci.x;
        ex = (M)(((uint64_t)ci.z << 32) | ci.y);
    }
    const uint4 *V = reinterpret_cast<const uint4 *>(base + v.recs) + 2 * first;
    while (m != 0) {
        const int k = W == 1 ? __ffs((unsigned)m) - 1 : __ffsll((unsigned long long)m) - 1;
        if (((ex >> k) & 1u) || filter_mismatch(s, d, sp, dp, V[2 * k], V[2 * k + 1], one) == 0u)
            return reinterpret_cast<const uint32_t *>(base + v.verdicts)[first + k];
        m &= m - 1;
    }
    return 0xFFFFFFFFu;
}

// First candidate of word w's AND m (record bits 32 w .. 32 w + 31 of class c's sub-list) that
// passes its exact test: its verdict word, or ~0u.
__device__ __forceinline__ uint32_t filter_word_first(const unsigned char *__restrict__ base, const FilterView &v,
                                                      const uint32_t *ex, const uint4 *V, int first, int w,
                                                      uint32_t m, uint32_t s, uint32_t d, uint32_t sp, uint32_t dp,
                                                      uint32_t one) {
    if (m == 0u) return 0xFFFFFFFFu;
    const uint32_t e = __ldg(ex + w);
    while (m != 0u) {
        const int k = 32 * w + __ffs(m) - 1;
        if (((e >> (k & 31)) & 1u) || filter_mismatch(s, d, sp, dp, __ldg(V + 2 * k), __ldg(V + 2 * k + 1), one) == 0u)
            return __ldg(reinterpret_cast<const uint32_t *>(base + v.verdicts) + first + k);
        m &= m - 1u;
    }
    return 0xFFFFFFFFu;
}

// Candidates of a packet of class c from word 0 on, given word 0's AND (m0), for
// any row width (v.words 32-bit words): each word's candidates are tested in
// order before the next word is read, so a packet reads its rows only up to its
// first match. Rows of kFilterSummaryMin words or more carry summaries (bit w:
// word w of the row is not zero); past word 0 a packet ANDs its three rows'
// summaries and reads only the words set in it, which include every word where
// the AND of the rows is not zero (a packet no rule matches often stops after
// the summaries).
// Returns the verdict word of the first match, or ~0u. The block is read
// through the L1 cache (global memory).
// SUMM: the rule set's rows carry summaries (v.words >= kFilterSummaryMin); without, every word
// up to the first match is read.
template <bool SUMM>
__device__ __forceinline__ uint32_t filter_resolve(const unsigned char *__restrict__ base, const FilterView &v,
                                                   uint32_t c, uint32_t s, uint32_t d, uint32_t sp, uint32_t dp,
                                                   uint32_t m0, uint32_t one) {
    const int W = v.words;
    const uint32_t *T = reinterpret_cast<const uint32_t *>(base + v.tables) + (size_t)c * 768u * W;
    const uint32_t *r0 = T + (s >> 24) * W;
    const uint32_t *r1 = T + (256u + (d >> 24)) * W;
    const uint32_t *r2 = T + (512u + (((sp >> 12) << 4) | (dp >> 12))) * W;
    const uint32_t *ex = reinterpret_cast<const uint32_t *>(base + v.exact) + (size_t)c * W;
    const int first = (int)__ldg(reinterpret_cast<const uint32_t *>(base + v.classes) + 4 * c);
    const uint4 *V = reinterpret_cast<const uint4 *>(base + v.recs) + 2 * first;
    if constexpr (!SUMM) {
        uint32_t m = m0;
        for (int w = 0; w < W; ++w) {
            if (w > 0) m = __ldg(r0 + w) & __ldg(r1 + w) & __ldg(r2 + w);
            if (m == 0u) continue;
            const uint32_t e = __ldg(ex + w);
            while (m != 0u) {
                const int k = 32 * w + __ffs(m) - 1;
                if (((e >> (k & 31)) & 1u) ||
                    filter_mismatch(s, d, sp, dp, __ldg(V + 2 * k), __ldg(V + 2 * k + 1), one) == 0u)
                    return __ldg(reinterpret_cast<const uint32_t *>(base + v.verdicts) + first + k);
                m &= m - 1u;
            }
        }
        return 0xFFFFFFFFu;
    } else {
        uint32_t vw = filter_word_first(base, v, ex, V, first, 0, m0, s, d, sp, dp, one);
        if (vw != 0xFFFFFFFFu) return vw;
        const int S = filter_summary_words(W);
        // the summaries follow the protocol class table (filter_layout)
        const uint32_t *Q = reinterpret_cast<const uint32_t *>(base + ((v.class_of + 256 + 15) & ~15)) +
                            (size_t)c * 768u * S;
        const uint32_t *q0 = Q + (s >> 24) * S;
        const uint32_t *q1 = Q + (256u + (d >> 24)) * S;
        const uint32_t *q2 = Q + (512u + (((sp >> 12) << 4) | (dp >> 12))) * S;
        for (int g = 0; g < S; ++g) {
            uint32_t sm = __ldg(q0 + g) & __ldg(q1 + g) & __ldg(q2 + g);
            if (g == 0) sm &= ~1u;  // word 0 is done
            while (sm != 0u) {
                const int w = 32 * g + __ffs(sm) - 1;
                sm &= sm - 1u;
                vw = filter_word_first(base, v, ex, V, first, w, __ldg(r0 + w) & __ldg(r1 + w) & __ldg(r2 + w), s, d,
                                       sp, dp, one);
                if (vw != 0xFFFFFFFFu) return vw;
            }
        }
        return 0xFFFFFFFFu;
    }
}

// Word 0 of the AND of a packet's three rows (class c), for any row width.
__device__ __forceinline__ uint32_t filter_word0(const unsigned char *__restrict__ base, const FilterView &v, uint32_t c,
                                                 uint32_t s, uint32_t d, uint32_t sp, uint32_t dp) {
    const uint32_t W = (uint32_t)v.words;
    const uint32_t *T = reinterpret_cast<const uint32_t *>(base + v.tables);
    const uint32_t cb = c * 768u;
    return __ldg(T + (cb + (s >> 24)) * W) & __ldg(T + (cb + 256u + (d >> 24)) * W) &
           __ldg(T + (cb + 512u + (((sp >> 12) << 4) | (dp >> 12))) * W);
}

// One packet, any row width, block read through L1 (SUMM: the rows carry summaries).
template <int KEY, bool SUMM>
__device__ __forceinline__ uint32_t filter_packet_wide(const unsigned char *__restrict__ base, const FilterView &v,
                                                       uint32_t s, uint32_t d, uint32_t sp, uint32_t dp, uint32_t pr,
                                                       uint32_t one) {
    const uint32_t c = filter_class<KEY>(base, v, s, d, pr);
    const uint32_t m0 = filter_word0(base, v, c, s, d, sp, dp);
    return SUMM ? filter_resolve<true>(base, v, c, s, d, sp, dp, m0, one)
                : filter_resolve<false>(base, v, c, s, d, sp, dp, m0, one);
}

// P packets of one lane, any row width, block read through L1 (every word up to the first match;
// the row summaries are left to the packet-split kernel, whose registers allow them): the classes and the
// first row words of all P packets are loaded before any candidate is tested, so
// those loads are in flight together; then each packet's candidates are tested in
// order. pr[] is overwritten with the classes; out[] gets the verdict words.
template <int P>
__device__ __forceinline__ void filter_packets_wide(const unsigned char *__restrict__ base, const FilterView &v,
                                                    const uint32_t (&s)[P], const uint32_t (&d)[P],
                                                    const uint32_t (&sp)[P], const uint32_t (&dp)[P], uint32_t (&pr)[P],
                                                    uint32_t one, uint32_t (&out)[P]) {
#pragma unroll
    for (int k = 0; k < P; ++k) pr[k] = filter_class<-1>(base, v, s[k], d[k], pr[k]);
#pragma unroll
    for (int k = 0; k < P; ++k) out[k] = filter_word0(base, v, pr[k], s[k], d[k], sp[k], dp[k]);
#pragma unroll
    for (int k = 0; k < P; ++k) out[k] = filter_resolve<false>(base, v, pr[k], s[k], d[k], sp[k], dp[k], out[k], one);
}

}  // namespace fwk
