// Internal definitions shared by the CUDA translation units of the library.
//
// Canonical device form of a rule (built once by fw_ruleset_create_ex):
//   match(p, r) = ((p.src ^ saddr) & smask) == 0         src prefix    (Sec. IV)
//               & ((p.dst ^ daddr) & dmask) == 0         dst prefix
//               & sport in [slo, shi] & dport in [dlo, dhi]   port ranges
//               & ((p.proto ^ pval) & pmask) == 0        proto, pmask 0 = any
// with saddr/daddr pre-masked and smask = 0 for prefix 0. Two equivalent
// encodings of the port test are kept:
//   clamp form:   ports = sport<<16 | dport, LO = slo<<16 | dlo, HI = shi<<16 | dhi;
//                 both ranges hold iff min16x2(max16x2(ports, LO), HI) == ports
//                 (per 16-bit lane, clamping a value into [lo, hi] leaves it
//                 unchanged exactly when it lies in the range);
//   compare form: (sport - slo) <= (shi - slo) as unsigned 32-bit, likewise dport
//                 (a port below slo wraps to a value above 2^32 - 65536).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fw.h"

namespace fwk {

constexpr int kChunkRules = 256;          // rules per TMA chunk / padding granule
constexpr int kMaxProtoClasses = 8;       // protocol classes: up to 7 exact protocols + "other"
// Classes of the partitioned rule lists (protocol class x address key). Eight,
// not more: on the 10K-rule list (4 protocol classes) one key bit, 8 classes,
// takes 0.243 ms against 0.273 with no key and 0.262 with two bits, 16 classes
// (the 100K-rule list: 5.37, 7.26 and 6.39 ms); past 8, more divergent groups
// and wider sort counters cost more than the shorter sub-lists save.
constexpr int kMaxClasses = 8;
constexpr uint32_t kStatusTimeout = 1u;   // a bounded wait gave up
constexpr uint32_t kStatusBadArgs = 2u;   // device-side sanity check failed

// Clamp-form record: 32 bytes = two uint4 (a: addresses, b: ports + proto).
struct RecClamp {
    uint4 a;  // saddr, smask, daddr, dmask
    uint4 b;  // LO, HI, pval, pmask
};

// Compare-form record: 48 bytes = three uint4.
struct RecCmp {
    uint4 a;  // saddr, smask, daddr, dmask
    uint4 b;  // slo, swidth, dlo, dwidth
    uint4 c;  // pval, pmask, 0, 0
};

// Arithmetic-form record: 32 bytes = two uint4, plus one word `wtop` per rule
// kept in a separate array (so that four rules' wtop words come in one 16-byte
// load). The port tests are written as unsigned subtractions that the FMA pipe can
// execute (IMAD), leaving only logic ops and compares on the ALU pipe:
//   sport:        (sport + neg_slo) <= swidth            (neg_slo = -slo mod 2^32)
//   dport, proto: (X * mul + add) <= wtop, X = proto << 17 | dport, where
//     exact proto p: mul = 1,      add = -(p << 17 | dlo), wtop = dhi - dlo
//     any proto:     mul = 2^15,   add = -(dlo << 15),      wtop = (dhi - dlo) << 15
//   With mul = 1 the protocol sits 17 bits above the port, so any protocol
//   difference moves the value at least 2^17 - 65535 > 65535 away from the
//   port window (or wraps it past 2^32 - 2^25); with mul = 2^15 the protocol
//   bits are shifted out of the 32-bit word and only the port difference,
//   scaled by 2^15, remains, which cannot wrap into the window.
struct RecArith {
    uint4 a;  // saddr, smask, daddr, dmask
    uint4 b;  // neg_slo, swidth, mul, add
};

// A record that no packet matches (used to pad the device arrays): its
// protocol value 0x100 differs from every 8-bit protocol under a full mask.
constexpr uint32_t kNeverProto = 0x100u;

struct Pkt {
    uint32_t src, dst, ports, proto;  // ports = sport << 16 | dport
};

__device__ __forceinline__ uint32_t ports_of(uint32_t sport, uint32_t dport) { return (sport << 16) | dport; }

// Non-zero exactly when the packet is outside the rule (clamp form).
__device__ __forceinline__ uint32_t mismatch_clamp(const Pkt &p, const uint4 &a, const uint4 &b) {
    uint32_t c = __vminu2(__vmaxu2(p.ports, b.x), b.y);
    return ((p.src ^ a.x) & a.y) | ((p.dst ^ a.z) & a.w) | (c ^ p.ports) | ((p.proto ^ b.z) & b.w);
}

// True exactly when the packet is inside the rule (compare form).
__device__ __forceinline__ bool match_cmp(const Pkt &p, const uint4 &a, const uint4 &b, const uint4 &c) {
    uint32_t mm = ((p.src ^ a.x) & a.y) | ((p.dst ^ a.z) & a.w) | ((p.proto ^ c.x) & c.y);
    uint32_t sp = p.ports >> 16, dp = p.ports & 0xFFFFu;
    return (mm == 0u) & ((sp - b.x) <= b.y) & ((dp - b.z) <= b.w);
}

// Packet form used with RecArith.
struct PktA {
    uint32_t src, dst, sport, x;  // x = proto << 17 | dport
};

__device__ __forceinline__ uint32_t x_of(uint32_t proto, uint32_t dport) { return (proto << 17) | dport; }

// True exactly when the packet is outside the rule (arithmetic form). `one`
// is the runtime constant 1, so that the sport subtraction is issued as a
// multiply-add on the FMA pipe instead of an add on the ALU pipe. The five
// field tests are one chain of predicated ALU operations: two 3-input logic
// ops (lop3 with LUT 0x28 = (a ^ b) & c) whose "result != 0" predicate is
// OR-ed into the chain, then two unsigned compares OR-ed into it.
__device__ __forceinline__ bool mismatch_arith(const PktA &p, const uint4 &a, const uint4 &b, uint32_t wtop,
                                               uint32_t one) {
    const uint32_t ts = p.sport * one + b.x;
    const uint32_t td = p.x * b.z + b.w;
    uint32_t r;
    asm("{\n\t"
        ".reg .pred q;\n\t"
        ".reg .b32 t;\n\t"
        "setp.ne.u32 q, 0, 0;\n\t"
        "lop3.or.b32 t|q, %1, %2, %3, 0x28, q;\n\t"
        "lop3.or.b32 t|q, %4, %5, %6, 0x28, q;\n\t"
        "setp.gt.or.u32 q, %7, %8, q;\n\t"
        "setp.gt.or.u32 q, %9, %10, q;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t"
        "}"
        : "=r"(r)
        : "r"(p.src), "r"(a.x), "r"(a.y), "r"(p.dst), "r"(a.z), "r"(a.w), "r"(ts), "r"(b.y), "r"(td), "r"(wtop));
    return r != 0u;
}

// Range-form record (32 bytes + one word in a separate array, like RecArith):
// every field test is "value - lo <= width" in unsigned 32-bit arithmetic, a
// prefix /len being the range [addr & mask, (addr & mask) + ~mask]:
//   a = {-src_lo, src_width, -dst_lo, dst_width}, b = {-sport_lo, swidth, mul, add},
//   wtop as in RecArith. Four multiply-adds (FMA pipe) produce the offsets and
//   four compares chained with .or (ALU pipe) give the mismatch predicate.
using RecRange = RecArith;

// Four rules at once, range form: non-zero exactly when the packet is outside
// all four. t[4k..4k+3] are rule k's four offsets, w[...] the four widths.
__device__ __forceinline__ uint32_t all_mismatch4_range(const uint32_t t[16], const uint32_t w[16]) {
    uint32_t r;
    asm("{\n\t"
        ".reg .pred q0, q1, q2, q3;\n\t"
        "setp.gt.u32 q0, %1, %2;\n\t"
        "setp.gt.or.u32 q0, %3, %4, q0;\n\t"
        "setp.gt.or.u32 q0, %5, %6, q0;\n\t"
        "setp.gt.or.u32 q0, %7, %8, q0;\n\t"
        "setp.gt.u32 q1, %9, %10;\n\t"
        "setp.gt.or.u32 q1, %11, %12, q1;\n\t"
        "setp.gt.or.u32 q1, %13, %14, q1;\n\t"
        "setp.gt.or.u32 q1, %15, %16, q1;\n\t"
        "setp.gt.u32 q2, %17, %18;\n\t"
        "setp.gt.or.u32 q2, %19, %20, q2;\n\t"
        "setp.gt.or.u32 q2, %21, %22, q2;\n\t"
        "setp.gt.or.u32 q2, %23, %24, q2;\n\t"
        "setp.gt.u32 q3, %25, %26;\n\t"
        "setp.gt.or.u32 q3, %27, %28, q3;\n\t"
        "setp.gt.or.u32 q3, %29, %30, q3;\n\t"
        "setp.gt.or.u32 q3, %31, %32, q3;\n\t"
        "and.pred q0, q0, q1;\n\t"
        "and.pred q2, q2, q3;\n\t"
        "and.pred q0, q0, q2;\n\t"
        "selp.u32 %0, 1, 0, q0;\n\t"
        "}"
        : "=r"(r)
        : "r"(t[0]), "r"(w[0]), "r"(t[1]), "r"(w[1]), "r"(t[2]), "r"(w[2]), "r"(t[3]), "r"(w[3]),
          "r"(t[4]), "r"(w[4]), "r"(t[5]), "r"(w[5]), "r"(t[6]), "r"(w[6]), "r"(t[7]), "r"(w[7]),
          "r"(t[8]), "r"(w[8]), "r"(t[9]), "r"(w[9]), "r"(t[10]), "r"(w[10]), "r"(t[11]), "r"(w[11]),
          "r"(t[12]), "r"(w[12]), "r"(t[13]), "r"(w[13]), "r"(t[14]), "r"(w[14]), "r"(t[15]), "r"(w[15]));
    return r;
}

__device__ __forceinline__ bool mismatch_range_c(const PktA &p, const uint4 &a, const uint4 &b, uint32_t wtop,
                                                 uint32_t one) {
    return ((p.src * one + a.x) > a.y) | ((p.dst * one + a.z) > a.w) | ((p.sport * one + b.x) > b.y) |
           ((p.x * b.z + b.w) > wtop);
}

// Partition class of a packet (see fw_ruleset): protocol class, then the top
// key_bits bits of the keyed address. key_shift = 32 - key_bits; with no key,
// key_field is 0 and the shift is never taken.
__device__ __forceinline__ uint32_t part_class(uint32_t pclass, int key_field, int key_bits, uint32_t src,
                                               uint32_t dst) {
    if (key_field == 0) return pclass;
    const uint32_t a = key_field == 1 ? src : dst;
    return (pclass << key_bits) | (a >> (32 - key_bits));
}

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared (TMA engine), completion signalled on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar` to complete, giving up after ~limit_ns.
// Returns false (and sets kStatusTimeout in *status) on give-up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned *status,
                                                  uint64_t limit_ns = 200000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && global_ns() - t0 > limit_ns) {
            atomicOr(status, kStatusTimeout);
            return false;
        }
    }
}

}  // namespace fwk

// Host-side view of a rule set (opaque to callers).
struct fw_ruleset {
    int64_t n;                // rules supplied
    int64_t n_eff;            // rules a scan can reach (first catch-all + 1, else n)
    int64_t n_pad;            // device array length: n_eff rounded up to kChunkRules (>= kChunkRules)
    int64_t first_catch_all;  // -1 if none
    int device;
    fwk::RecClamp *d_clamp;   // n_pad records
    fwk::RecCmp *d_cmp;       // n_pad records
    fwk::RecArith *d_arith;   // n_pad records
    uint32_t *d_wtop;         // n_pad words (arithmetic form)
    fwk::RecArith *d_range;   // n_pad records (range form)
    uint32_t *d_range_wtop;   // n_pad words (range form)
    // Partition (arithmetic form): a packet's class is its protocol class
    // (d_class_of) times 2^key_bits plus the top key_bits bits of its source
    // (key_field 1) or destination (key_field 2) address. Class c's sub-list
    // holds, in list order, the reachable rules that can contain a packet of
    // class c; the sub-lists are stored one after another.
    int32_t n_classes;                 // 1..kMaxClasses (protocol classes << key_bits)
    int32_t key_field;                 // 0 = no address key, 1 = src, 2 = dst
    int32_t key_bits;                  // 0..3
    int32_t class_off[fwk::kMaxClasses];  // first record of each sub-list (multiple of 4)
    int32_t class_len[fwk::kMaxClasses];  // records in each sub-list (multiple of 4, padding never matches)
    int64_t part_pad;                  // records stored (multiple of kChunkRules)
    uint8_t *d_class_of;               // 256 entries: protocol -> protocol class
    fwk::RecArith *d_part;             // part_pad records
    uint32_t *d_part_wtop;             // part_pad words
    int32_t *d_part_orig;              // part_pad original rule indices (-1 for padding)
    uint32_t *d_part_verdict;          // part_pad words: original index | action << 31
    // Bucket filter over the partition (fw_filter.cuh): per class, bitmaps over
    // the class sub-list indexed by a packet's address and port buckets, plus an
    // exact-test record per stored record. Built when every sub-list holds at
    // most kFilterMaxRecords records and no class mixes exact protocols.
    int32_t filter_words;              // 0 = no filter, else 32-bit words per bitmap row
    int64_t filter_bytes;              // bytes of d_filter
    unsigned char *d_filter;           // the filter block (layout: FilterLayout)
    uint8_t *d_action;        // n_pad actions
    unsigned *d_status;       // device error flags (kStatus*)
};

namespace fwk {
int set_status(int s);  // records s as this thread's last status; returns s
// FW_OK when the current device is the one the rule set was created on, FW_EINVAL
// when it is another, FW_ECUDA when the current device cannot be read.
int check_device(const fw_ruleset *rs);
int cuda_status(cudaError_t e);
uint32_t prefix_mask(unsigned prefix);  // top `prefix` bits set; 0 for prefix 0
bool is_catch_all(const fw_rule &r);    // all five fields wildcards
int validate_rule(const fw_rule &r);    // FW_OK or FW_EINVAL
// Protocol partition of rules [0, n): up to kMaxProtoClasses - 1 classes for the
// exact protocols those rules use most, plus "other" for every other protocol
// value. class_of[p] is protocol p's class; lists[c] holds, in list order, the
// rules whose protocol set can contain a packet of class c (protocol "any", or
// class c's protocol; for "other": any, or an exact protocol without a class).
void protocol_classes(const fw_rule *rules, int64_t n, std::vector<uint8_t> &class_of,
                      std::vector<std::vector<int64_t>> &lists);
// Partition of rules [0, n) into the classes the packet-split and learned-index
// kernels use: protocol classes as above, each split again by the top key_bits
// bits of the source (key_field 1) or destination (2) address; key_field 0 is
// no key. Class c = pclass << key_bits | key, and lists[c] keeps, in list
// order, the rules of pclass's list whose address prefix on that field can
// contain an address with top bits `key` (a prefix shorter than key_bits covers
// several keys; prefix 0 covers all). So a packet's list holds every rule that
// can match it, in order, and its first match is unchanged. The key (at most
// kMaxClasses classes in all) is the one with the lowest mean list cost, what a
// packet scans when key values are spread evenly: the length (granule <= 1),
// else ceil(length / granule) with a minimum of 1, for a reader that takes the
// list `granule` rules at a time. No key when none lowers it or the protocols
// alone fill the classes.
void partition_lists(const fw_rule *rules, int64_t n, int64_t granule, std::vector<uint8_t> &class_of,
                     std::vector<std::vector<int64_t>> &lists, int &key_field, int &key_bits);
int sm_count(int dev);                  // SMs of device `dev` (cached)

// Bucket filter (fw_filter.cu). Byte offsets of the parts of the filter block
// for n_classes classes, `words` 32-bit words per bitmap row and `records`
// stored sub-list records (every part starts on a 16-byte boundary).
struct FilterLayout {
    int64_t tables, classes, exact, recs, verdicts, class_of, summary, total;
};
// Summary words per bitmap row: rows of at least kFilterSummaryMin words carry, after the rest of
// the block, a summary of ceil(W / 32) words per row whose bit w is set when word w of the row is
// not zero. (On 95-word rows reading the summaries first took a classification from 3.36 to 2.31
// ms; on 9-word rows, most of whose words are not zero, it cost a quarter more time.)
constexpr int kFilterSummaryMin = 32;
__host__ __device__ inline int filter_summary_words(int words) {
    return words >= kFilterSummaryMin ? (words + 31) / 32 : 0;
}
constexpr int kFilterTables = 3;  // source top 8 bits, destination top 8 bits, (sport, dport) top 4 bits each
constexpr int kFilterMaxRecords = FW_FILTER_MAX_RULES;  // longest class sub-list a filter covers
__host__ __device__ inline FilterLayout filter_layout(int n_classes, int words, int64_t records) {
    FilterLayout L;
    auto up16 = [](int64_t b) { return (b + 15) / 16 * 16; };
    L.tables = 0;                                                          // [class][table][256][words] uint32
    L.classes = up16(L.tables + (int64_t)kFilterTables * n_classes * 256 * words * 4);  // [class] uint4
    L.exact = L.classes + (int64_t)n_classes * 16;                         // [class][words] uint32
    L.recs = up16(L.exact + (int64_t)n_classes * words * 4);               // [record] 2 x uint4
    L.verdicts = L.recs + records * 32;                                    // [record] uint32
    L.class_of = up16(L.verdicts + records * 4);                           // [256] uint8
    L.summary = up16(L.class_of + 256);  // W >= kFilterSummaryMin: [class][table][256][ceil(W / 32)] uint32
    L.total = L.summary + (int64_t)kFilterTables * n_classes * 256 * filter_summary_words(words) * 4;
    return L;
}
// Builds rs->d_filter from the partition (lists[c] = original rule indices of
// class c's sub-list, class_of = protocol -> protocol class) when it applies;
// leaves filter_words 0 otherwise. Returns a CUDA error only for a failed
// allocation or copy.
cudaError_t build_filter(const fw_rule *rules, const std::vector<std::vector<int64_t>> &lists,
                         const std::vector<uint8_t> &class_of, fw_ruleset *rs);
// The filter block itself (host only): fills `blk` and returns the words per bitmap row, or
// returns 0 (and leaves `blk` empty) when the partition does not admit a filter.
int filter_block(const fw_rule *rules, const std::vector<std::vector<int64_t>> &lists,
                 const std::vector<uint8_t> &class_of, int key_bits, const int32_t *class_off,
                 const int32_t *class_len, std::vector<unsigned char> &blk);
// Offsets and lengths of the stored sub-lists: each list padded to a multiple of 4 records,
// stored one after another (kMaxClasses entries; classes past lists.size() are empty).
void pack_sublists(const std::vector<std::vector<int64_t>> &lists, int32_t *class_off, int32_t *class_len);
struct HdrPtrs;
// Rule split (fw_rule_split.cu): warp, block or grid mode over the partition or the whole
// list; grid mode combines through `scratch` (n int32 of device memory) when it is given, else
// through a stream-ordered allocation.
int rule_split_run(const fw_ruleset *rs, const HdrPtrs &h, int64_t n, int32_t *out_idx, uint8_t *out_act,
                   cudaStream_t st, const fw_config &cfg, int32_t *scratch);
int launch_rule_split(const fw_ruleset *rs, const HdrPtrs &h, int64_t n, int32_t *out_idx, uint8_t *out_act,
                      cudaStream_t st, const fw_config &cfg);
// Packet split through the bucket filter (FW_OK, or a status for a bad
// configuration / launch failure). threads, blocks_per_sm, lane_packets (packets per
// thread per step, 2 or 4): launch shape (0 = default).
int launch_filter(const fw_ruleset *rs, const HdrPtrs &h, int64_t n, int32_t *out_idx, uint8_t *out_act,
                  cudaStream_t st, int threads, int blocks_per_sm, int lane_packets);
}  // namespace fwk
