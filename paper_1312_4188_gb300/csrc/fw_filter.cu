// Packet split through a bucket filter (Sec. IV.A data-parallel: every thread
// holds the whole rule list and takes its own packets; first match, default
// deny, Sec. I).
//
// The rule list is partitioned as for the other packet-split kernels: a packet
// of class c (its protocol class and address key) can only be matched by the
// rules of class c's sub-list, kept in list order. For sub-lists of at most
// 512 records each class also gets three bitmaps per bucket value, one bit per
// sub-list record:
//   table 0, bucket = top 8 bits of the source address: bit j set when rule j's
//            source prefix contains some address with those top bits;
//   table 1, the same for the destination address;
//   table 2, bucket = (sport >> 12) << 4 | (dport >> 12): bit j set when rule
//            j's source port range meets [sb*4096, sb*4096+4095] and its
//            destination port range meets [db*4096, db*4096+4095].
// A rule that contains the packet passes all three (each of its field sets
// holds the packet's value, so it meets the bucket of that value), so the AND
// of the packet's three rows is a superset of the sub-list rules that match
// it. Testing the candidates in increasing bit order, exactly, and stopping at
// the first that passes therefore returns the first match of the sub-list,
// which is the packet's first match in the whole list. A candidate whose
// fields are unions of whole buckets (prefixes of at most 8 bits, port ranges
// aligned to 4,096) passes exactly when its bits are set, so it needs no test
// (the exact mask; the catch-all is one such rule).
//
// The exact test reads one 32-byte record per candidate, the arithmetic form
// of the address and port tests: {saddr & smask, smask, daddr & dmask,
// dmask} and {-sport_lo, sport_hi - sport_lo, -dport_lo, dport_hi - dport_lo}
// (mod 2^32); the addresses are tested as ((a ^ addr) & mask) == 0 with one
// 3-input logic op each, the ports as (port - lo) <= width with one
// multiply-add (FMA pipe) and one unsigned compare each, all four chained into
// one predicate.
// The protocol needs no test: every rule of an exact-protocol class has that
// protocol or "any", and the filter is built only when the "every other
// protocol" class holds no exact-protocol rule.
//
// One filter block (tables, class info, exact masks, records, verdict words,
// the protocol class table). Rows of one or two words: every block stages the
// filter block into its shared memory by 1-D TMA bulk copies (no multicast)
// with a bounded mbarrier wait, and a row is one integer. Wider rows (sub-lists
// of 65..512 records): the block stays in global memory, read through L1, and
// the rows are ANDed a word at a time up to the first match. In both, a thread
// takes four consecutive packets per step (16-byte header loads), so a warp
// streams 832 contiguous header bytes per step and writes its verdicts with
// 16-byte and 4-byte stores.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "fw_alloc.h"
#include "fw_filter.cuh"

namespace fwk {

struct FilterParams {
    const unsigned char *blk;  // the filter block in global memory
    FilterView v;
    int32_t blk_bytes;
    uint32_t one;  // the constant 1, opaque to the compiler (the port offsets become multiply-adds)
    HdrPtrs h;
    int64_t n;
    int32_t *out_idx;
    uint8_t *out_act;
    unsigned *status;
};

// Verdict word of one packet (~0u when no rule matches). W = 1, 2: one-integer
// rows from `base` (shared memory); W = 0: rows of any width from global memory;
// W = -1: the same, rows with summaries.
template <int W, int KEY>
__device__ __forceinline__ uint32_t filter_verdict(const unsigned char *base, const FilterParams &p, uint32_t s,
                                                   uint32_t d, uint32_t sp, uint32_t dp, uint32_t pr) {
    if constexpr (W <= 0) {
        return filter_packet_wide<KEY, (W < 0)>(base, p.v, s, d, sp, dp, pr, p.one);
    } else {
        uint32_t cls;
        const FilterMask<W> m = filter_candidates<W, KEY>(base, p.v, s, d, sp, dp, pr, cls);
        return filter_first<W>(base, p.v, m, cls, s, d, sp, dp, p.one);
    }
}

// The grid-stride loop over packet quads, with the filter block at `base`
// (shared memory, or global memory after a failed staging wait).
template <int W, int KEY, bool VEC>
__device__ __forceinline__ void filter_loop(const FilterParams &p, const unsigned char *base) {
    const int64_t nq = (p.n + 3) / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += stride) {
        uint32_t s[4], d[4], sp[4], dp[4], pr[4];
        int cnt = 4;
        const int64_t b = q * 4;
        if (VEC && b + 3 < p.n) {
            const uint4 sv = __ldcs(reinterpret_cast<const uint4 *>(p.h.src) + q);
            const uint4 dv = __ldcs(reinterpret_cast<const uint4 *>(p.h.dst) + q);
            const uint2 spv = __ldcs(reinterpret_cast<const uint2 *>(p.h.sport) + q);
            const uint2 dpv = __ldcs(reinterpret_cast<const uint2 *>(p.h.dport) + q);
            const uint32_t prv = __ldcs(reinterpret_cast<const unsigned int *>(p.h.proto) + q);
            s[0] = sv.x, s[1] = sv.y, s[2] = sv.z, s[3] = sv.w;
            d[0] = dv.x, d[1] = dv.y, d[2] = dv.z, d[3] = dv.w;
            sp[0] = spv.x & 0xFFFFu, sp[1] = spv.x >> 16, sp[2] = spv.y & 0xFFFFu, sp[3] = spv.y >> 16;
            dp[0] = dpv.x & 0xFFFFu, dp[1] = dpv.x >> 16, dp[2] = dpv.y & 0xFFFFu, dp[3] = dpv.y >> 16;
#pragma unroll
            for (int j = 0; j < 4; ++j) pr[j] = (prv >> (8 * j)) & 0xFFu;
        } else {
            cnt = p.n - b < 4 ? (int)(p.n - b) : 4;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const bool in = j < cnt;
                s[j] = in ? p.h.src[b + j] : 0u;
                d[j] = in ? p.h.dst[b + j] : 0u;
                sp[j] = in ? p.h.sport[b + j] : 0u;
                dp[j] = in ? p.h.dport[b + j] : 0u;
                pr[j] = in ? p.h.proto[b + j] : 0u;
            }
        }
        int32_t idx[4];
        uint32_t acts = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t vw = filter_verdict<W, KEY>(base, p, s[j], d[j], sp[j], dp[j], pr[j]);
            idx[j] = vw == 0xFFFFFFFFu ? -1 : (int32_t)(vw & 0x7FFFFFFFu);
            acts |= (vw == 0xFFFFFFFFu ? (uint32_t)FW_DROP : vw >> 31) << (8 * j);
        }
        if (VEC && cnt == 4) {
            __stcs(reinterpret_cast<int4 *>(p.out_idx) + q, make_int4(idx[0], idx[1], idx[2], idx[3]));
            __stcs(reinterpret_cast<unsigned int *>(p.out_act) + q, acts);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j < cnt) {
                    p.out_idx[b + j] = idx[j];
                    p.out_act[b + j] = (uint8_t)(acts >> (8 * j));
                }
            }
        }
    }
}

// The same loop over packet pairs (8-byte, 4-byte and 2-byte header loads): half the header
// registers of the quad loop, so four 512-thread blocks fit on an SM.
template <int W, int KEY, bool VEC>
__device__ __forceinline__ void filter_loop_pairs(const FilterParams &p, const unsigned char *base) {
    const int64_t np = (p.n + 1) / 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += stride) {
        uint32_t s[2], d[2], sp[2], dp[2], pr[2];
        const int64_t b = q * 2;
        const bool full = b + 1 < p.n;
        if (VEC && full) {
            const uint2 sv = __ldcs(reinterpret_cast<const uint2 *>(p.h.src) + q);
            const uint2 dv = __ldcs(reinterpret_cast<const uint2 *>(p.h.dst) + q);
            const uint32_t spv = __ldcs(reinterpret_cast<const unsigned int *>(p.h.sport) + q);
            const uint32_t dpv = __ldcs(reinterpret_cast<const unsigned int *>(p.h.dport) + q);
            const uint32_t prv = __ldcs(reinterpret_cast<const unsigned short *>(p.h.proto) + q);
            s[0] = sv.x, s[1] = sv.y, d[0] = dv.x, d[1] = dv.y;
            sp[0] = spv & 0xFFFFu, sp[1] = spv >> 16, dp[0] = dpv & 0xFFFFu, dp[1] = dpv >> 16;
            pr[0] = prv & 0xFFu, pr[1] = prv >> 8;
        } else {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const bool in = b + j < p.n;
                s[j] = in ? p.h.src[b + j] : 0u;
                d[j] = in ? p.h.dst[b + j] : 0u;
                sp[j] = in ? p.h.sport[b + j] : 0u;
                dp[j] = in ? p.h.dport[b + j] : 0u;
                pr[j] = in ? p.h.proto[b + j] : 0u;
            }
        }
        int32_t idx[2];
        uint32_t acts = 0;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const uint32_t vw = filter_verdict<W, KEY>(base, p, s[j], d[j], sp[j], dp[j], pr[j]);
            idx[j] = vw == 0xFFFFFFFFu ? -1 : (int32_t)(vw & 0x7FFFFFFFu);
            acts |= (vw == 0xFFFFFFFFu ? (uint32_t)FW_DROP : vw >> 31) << (8 * j);
        }
        if (VEC && full) {
            __stcs(reinterpret_cast<int2 *>(p.out_idx) + q, make_int2(idx[0], idx[1]));
            __stcs(reinterpret_cast<unsigned short *>(p.out_act) + q, (unsigned short)acts);
        } else {
            for (int j = 0; j < 2; ++j) {
                if (b + j < p.n) {
                    p.out_idx[b + j] = idx[j];
                    p.out_act[b + j] = (uint8_t)(acts >> (8 * j));
                }
            }
        }
    }
}

// Stage the filter block into shared memory (1-D TMA bulk copies, one bounded mbarrier wait);
// false when the wait gave up.
__device__ __forceinline__ bool filter_stage(const FilterParams &p, unsigned char *smem, uint64_t *bar) {
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, (uint32_t)p.blk_bytes);
        for (int32_t o = 0; o < p.blk_bytes; o += 32768)
            bulk_load(smem + o, p.blk + o, (uint32_t)min(32768, p.blk_bytes - o), bar);
    }
    const bool ok = mbar_wait_bounded(bar, 0, p.status);
    return __syncthreads_and(ok) != 0;
}

template <int W, int KEY, bool VEC>
__global__ void __launch_bounds__(512, 4) k_packet_split_filter_pairs(FilterParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    if (filter_stage(p, smem, &bar)) {
        filter_loop_pairs<W, KEY, VEC>(p, smem);
    } else {
        filter_loop_pairs<W, KEY, VEC>(p, p.blk);
        if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, p.status);
    }
}

template <int W, int KEY, bool VEC>
__global__ void __launch_bounds__(512, 3) k_packet_split_filter(FilterParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    if (filter_stage(p, smem, &bar)) {
        filter_loop<W, KEY, VEC>(p, smem);
    } else {
        // a failed wait leaves the block reading the filter from global memory; before it exits,
        // the copies that may still be in flight into its shared memory get a second bounded wait
        filter_loop<W, KEY, VEC>(p, p.blk);
        if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, p.status);
    }
}

// Rows wider than two words: the filter block is read from global memory (L1); SUMM: the rows
// carry summaries.
template <int KEY, bool VEC, bool SUMM>
__global__ void __launch_bounds__(512, SUMM ? 2 : 3) k_packet_split_filter_wide(FilterParams p) {
    filter_loop<SUMM ? -1 : 0, KEY, VEC>(p, p.blk);
}

// ------------------------------------------------------------ host side
// Exact-test record of a rule (layout above).
static void verify_record(const fw_rule &r, uint4 *rec) {
    const uint32_t sm = prefix_mask(r.src_prefix), dm = prefix_mask(r.dst_prefix);
    rec[0] = make_uint4(r.src_addr & sm, sm, r.dst_addr & dm, dm);
    rec[1] = make_uint4(0u - (uint32_t)r.sport_lo, (uint32_t)(r.sport_hi - r.sport_lo), 0u - (uint32_t)r.dport_lo,
                        (uint32_t)(r.dport_hi - r.dport_lo));
}

// Does the prefix (addr, len) contain an address whose top 8 bits are b?
static bool prefix_meets_bucket(uint32_t addr, unsigned len, uint32_t b) {
    if (len == 0) return true;
    if (len >= 8) return (addr >> 24) == b;
    return (b >> (8 - len)) == (addr >> (32 - len));
}

int filter_block(const fw_rule *rules, const std::vector<std::vector<int64_t>> &lists,
                 const std::vector<uint8_t> &class_of, int key_bits, const int32_t *class_off,
                 const int32_t *class_len, std::vector<unsigned char> &blk) {
    blk.clear();
    const int nc = (int)lists.size();
    const int n_proto_classes = nc >> key_bits;
    int longest = 0;
    for (int c = 0; c < nc; ++c) longest = std::max(longest, class_len[c]);
    if (nc < 1 || longest > kFilterMaxRecords) return 0;
    // the "every other protocol" classes must hold protocol-"any" rules only
    for (int c = 0; c < nc; ++c) {
        if ((c >> key_bits) != n_proto_classes - 1) continue;
        for (int64_t k : lists[c])
            if (!rules[k].proto_any) return 0;
    }
    const int W = (longest + 31) / 32 > 0 ? (longest + 31) / 32 : 1;
    const int64_t records = class_off[kMaxClasses - 1] + class_len[kMaxClasses - 1];
    const FilterLayout L = filter_layout(nc, W, records);
    blk.assign((size_t)L.total, 0);
    uint32_t *tab = reinterpret_cast<uint32_t *>(blk.data() + L.tables);
    uint4 *cinfo = reinterpret_cast<uint4 *>(blk.data() + L.classes);
    uint32_t *exact_all = reinterpret_cast<uint32_t *>(blk.data() + L.exact);
    uint4 *recs = reinterpret_cast<uint4 *>(blk.data() + L.recs);
    uint32_t *vw = reinterpret_cast<uint32_t *>(blk.data() + L.verdicts);
    auto set_bit = [&](uint32_t *row, int j) { row[j >> 5] |= 1u << (j & 31); };
    auto row = [&](int c, int t, uint32_t b) { return tab + (((size_t)c * kFilterTables + t) * 256 + b) * W; };
    for (int c = 0; c < nc; ++c) {
        uint32_t *exact = exact_all + (size_t)c * W;
        for (size_t j = 0; j < lists[c].size(); ++j) {
            const fw_rule &r = rules[lists[c][j]];
            const int64_t at = class_off[c] + (int64_t)j;
            verify_record(r, recs + 2 * at);
            vw[at] = (uint32_t)lists[c][j] | ((uint32_t)(r.action & 1u) << 31);
            for (uint32_t b = 0; b < 256; ++b) {
                if (prefix_meets_bucket(r.src_addr, r.src_prefix, b)) set_bit(row(c, 0, b), (int)j);
                if (prefix_meets_bucket(r.dst_addr, r.dst_prefix, b)) set_bit(row(c, 1, b), (int)j);
            }
            for (uint32_t sb = (uint32_t)r.sport_lo >> 12; sb <= (uint32_t)r.sport_hi >> 12; ++sb)
                for (uint32_t db = (uint32_t)r.dport_lo >> 12; db <= (uint32_t)r.dport_hi >> 12; ++db)
                    set_bit(row(c, 2, (sb << 4) | db), (int)j);
            const bool whole = r.src_prefix <= 8 && r.dst_prefix <= 8 && (r.sport_lo & 0xFFFu) == 0 &&
                               (r.sport_hi & 0xFFFu) == 0xFFFu && (r.dport_lo & 0xFFFu) == 0 &&
                               (r.dport_hi & 0xFFFu) == 0xFFFu;
            if (whole) exact[j >> 5] |= 1u << (j & 31);
        }
        cinfo[c] = make_uint4((uint32_t)class_off[c], exact[0], W > 1 ? exact[1] : 0u, 0u);
        // summaries of wide rows: bit w of a row's summary set when its word w is not zero
        const int S = filter_summary_words(W);
        if (S > 0) {
            uint32_t *summ = reinterpret_cast<uint32_t *>(blk.data() + L.summary);
            for (int t = 0; t < kFilterTables; ++t)
                for (uint32_t b = 0; b < 256; ++b) {
                    const uint32_t *rw = row(c, t, b);
                    uint32_t *sw = summ + (((size_t)c * kFilterTables + t) * 256 + b) * S;
                    for (int w = 0; w < W; ++w)
                        if (rw[w] != 0u) sw[w >> 5] |= 1u << (w & 31);
                }
        }
    }
    std::memcpy(blk.data() + L.class_of, class_of.data(), 256);
    return W;
}

cudaError_t build_filter(const fw_rule *rules, const std::vector<std::vector<int64_t>> &lists,
                         const std::vector<uint8_t> &class_of, fw_ruleset *rs) {
    rs->filter_words = 0;
    rs->filter_bytes = 0;
    rs->d_filter = nullptr;
    std::vector<unsigned char> blk;
    const int W = filter_block(rules, lists, class_of, rs->key_bits, rs->class_off, rs->class_len, blk);
    if (W == 0) return cudaSuccess;
    cudaError_t e = dev_malloc(&rs->d_filter, blk.size());
    if (e == cudaSuccess) e = cudaMemcpy(rs->d_filter, blk.data(), blk.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    rs->filter_words = W;
    rs->filter_bytes = (int64_t)blk.size();
    return cudaSuccess;
}

// Shared-memory staging applies to rows of one or two words whose block fits three blocks per SM.
bool filter_staged(const fw_ruleset *rs) { return rs->filter_words <= 2 && rs->filter_bytes <= 72 * 1024; }

int launch_filter(const fw_ruleset *rs, const HdrPtrs &h, int64_t n, int32_t *out_idx, uint8_t *out_act,
                  cudaStream_t st, int threads, int blocks_per_sm, int lane_packets) {
    if (rs->filter_words == 0) return FW_EINVAL;
    FilterParams p;
    std::memset(&p, 0, sizeof(p));
    p.blk = rs->d_filter;
    p.v = filter_view(rs);
    p.blk_bytes = (int32_t)rs->filter_bytes;
    p.one = 1u;
    p.h = h;
    p.n = n;
    p.out_idx = out_idx;
    p.out_act = out_act;
    p.status = rs->d_status;
    const bool staged = filter_staged(rs);
    if (lane_packets != 0 && lane_packets != 2 && lane_packets != 4) return FW_EINVAL;
    // two packets per thread, four blocks per SM: on request, and by default for batches under 2^20
    // packets, which four packets per thread spread over too few blocks (1,000 rules x 100,000
    // packets, L2 flushed: 8.19 against 8.93-9.95 us per launch); larger batches take four (the
    // 10K x 16M step: 241 against 234 Gpackets/s)
    const bool pairs = staged && (lane_packets == 2 || (lane_packets == 0 && n < (int64_t(1) << 20)));
    const size_t smem = staged ? (size_t)rs->filter_bytes : 0;
    // Default shape: three 512-thread blocks per SM (1,536 threads, 40 registers each), fewer
    // when their shared memory does not fit; two packets per thread: four blocks. On the 10K x 16M
    // step, 256 x 6, 384 x 4 and 512 x 3 measure the same (241 Gpackets/s back to back).
    threads = threads > 0 ? threads : 512;
    if (threads % 32 != 0 || threads > 512 || blocks_per_sm > 64) return FW_EINVAL;
    // (the wide kernel with row summaries holds two 512-thread blocks per SM)
    const bool summ = !staged && rs->filter_words >= kFilterSummaryMin;
    int per_sm = blocks_per_sm > 0 ? blocks_per_sm : (pairs ? 4 : summ ? 2 : 3);
    if (blocks_per_sm <= 0)
        while (per_sm > 1 && (size_t)per_sm * (smem + 1024) > 228 * 1024) --per_sm;
    if (staged && (size_t)per_sm * (smem + 1024) > 228 * 1024) return FW_EINVAL;
    const int64_t nq = pairs ? (n + 1) / 2 : (n + 3) / 4;
    int64_t blocks = std::min<int64_t>((int64_t)sm_count(rs->device) * per_sm, (nq + threads - 1) / threads);
    blocks = std::max<int64_t>(1, blocks);
    // vector loads: a quad's (or pair's) header fields and verdicts each in one aligned access
    const int u = pairs ? 2 : 4;
    auto al = [](const void *q, size_t a) { return reinterpret_cast<uintptr_t>(q) % a == 0; };
    const bool vec = al(h.src, 4 * u) && al(h.dst, 4 * u) && al(h.sport, 2 * u) && al(h.dport, 2 * u) &&
                     al(h.proto, u) && al(out_idx, 4 * u) && al(out_act, u);
    const int key = p.v.key_field;
    cudaError_t e = cudaSuccess;
#define FW_LAUNCH_F(WW, KK, V)                                                                              \
    do {                                                                                                    \
        if (pairs) {                                                                                        \
            if (smem > 48 * 1024)                                                                           \
                e = cudaFuncSetAttribute(k_packet_split_filter_pairs<WW, KK, V>,                            \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);           \
            if (e == cudaSuccess)                                                                           \
                k_packet_split_filter_pairs<WW, KK, V><<<(unsigned)blocks, threads, smem, st>>>(p);         \
        } else {                                                                                            \
            if (smem > 48 * 1024)                                                                           \
                e = cudaFuncSetAttribute(k_packet_split_filter<WW, KK, V>,                                  \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);           \
            if (e == cudaSuccess) k_packet_split_filter<WW, KK, V><<<(unsigned)blocks, threads, smem, st>>>(p); \
        }                                                                                                   \
    } while (0)
#define FW_LAUNCH_G(KK, V)                                                                                  \
    do {                                                                                                    \
        if (rs->filter_words >= kFilterSummaryMin)                                                         \
            k_packet_split_filter_wide<KK, V, true><<<(unsigned)blocks, threads, 0, st>>>(p);              \
        else                                                                                                \
            k_packet_split_filter_wide<KK, V, false><<<(unsigned)blocks, threads, 0, st>>>(p);             \
    } while (0)
#define FW_LAUNCH_FK(WW, V)                                                                                 \
    do {                                                                                                    \
        if (!staged) {                                                                                      \
            if (key == 1) FW_LAUNCH_G(1, V);                                                                \
            else if (key == 2) FW_LAUNCH_G(2, V);                                                           \
            else FW_LAUNCH_G(0, V);                                                                         \
        } else if (key == 1) FW_LAUNCH_F(WW, 1, V);                                                         \
        else if (key == 2) FW_LAUNCH_F(WW, 2, V);                                                           \
        else FW_LAUNCH_F(WW, 0, V);                                                                         \
    } while (0)
    if (rs->filter_words == 1) {
        if (vec) FW_LAUNCH_FK(1, true);
        else FW_LAUNCH_FK(1, false);
    } else {
        if (vec) FW_LAUNCH_FK(2, true);
        else FW_LAUNCH_FK(2, false);
    }
#undef FW_LAUNCH_FK
#undef FW_LAUNCH_G
#undef FW_LAUNCH_F
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(cudaGetLastError());
}

}  // namespace fwk

using namespace fwk;

extern "C" int fw_filter_plan(const fw_rule *rules, int64_t n, void *block, int64_t capacity, int64_t *bytes,
                              int32_t *words, int32_t *class_off, int32_t *class_len) {
    if (n < 0 || (n > 0 && rules == nullptr) || n > (int64_t(1) << 30) || capacity < 0 ||
        (capacity > 0 && block == nullptr) || bytes == nullptr || words == nullptr)
        return set_status(FW_EINVAL);
    int64_t n_eff = n;
    for (int64_t k = 0; k < n; ++k) {
        const int s = validate_rule(rules[k]);
        if (s != FW_OK) return set_status(s);
        if (n_eff == n && is_catch_all(rules[k])) n_eff = k + 1;
    }
    std::vector<uint8_t> class_of;
    std::vector<std::vector<int64_t>> lists;
    int key_field = 0, key_bits = 0;
    partition_lists(rules, n_eff, 1, class_of, lists, key_field, key_bits);
    int32_t off[kMaxClasses], len[kMaxClasses];
    pack_sublists(lists, off, len);
    std::vector<unsigned char> blk;
    *words = filter_block(rules, lists, class_of, key_bits, off, len, blk);
    *bytes = (int64_t)blk.size();
    if (class_off != nullptr) std::memcpy(class_off, off, sizeof(off));
    if (class_len != nullptr) std::memcpy(class_len, len, sizeof(len));
    if (!blk.empty() && capacity > 0) {
        if (capacity < (int64_t)blk.size()) return set_status(FW_ERANGE);
        std::memcpy(block, blk.data(), blk.size());
    }
    return FW_OK;
}
