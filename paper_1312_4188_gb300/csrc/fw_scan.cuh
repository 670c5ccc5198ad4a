// Record policies, packet loads and rule-scan helpers shared by the scan
// kernels (fw_scan.cu) and the batched persistent kernel (fw_batch.cu).
#pragma once

#include <type_traits>

#include "fw_internal.cuh"

namespace fwk {

struct HdrPtrs {
    const uint32_t *src;
    const uint32_t *dst;
    const uint16_t *sport;
    const uint16_t *dport;
    const uint8_t *proto;
};

struct ScanParams {
    const void *rec;       // records of the chosen form (RecClamp / RecCmp / RecArith)
    const uint32_t *wtop;  // arithmetic form: per-rule wtop words
    const uint8_t *action;
    int n_scan;   // rules scanned: n_eff rounded up to a multiple of 4 (padding never matches)
    int n_smem;   // rules resident in shared memory (multiple of kChunkRules, <= n_pad)
    int batch;    // compacting kernel: packets per warp batch (multiple of 128)
    int seg0;     // compacting kernel: rules in the first segment (multiple of 4)
    uint32_t one; // the constant 1, opaque to the compiler (see mismatch_arith)
    HdrPtrs h;
    int64_t n;
    int32_t *out_idx;
    uint8_t *out_act;
    unsigned *status;
    // protocol partition (used by the PART kernels; records are then the
    // concatenated sub-lists and n_scan / n_smem refer to that array)
    int32_t n_classes;
    int32_t key_field, key_bits;  // address key of the partition (see part_class)
    int32_t class_off[kMaxClasses];
    int32_t class_len[kMaxClasses];
    const uint8_t *class_of;  // 256 entries: protocol -> protocol class
    const int32_t *orig;      // original rule index of each stored record
    const uint32_t *verdict;  // the same index | action << 31 (one load per decided packet)
};

// ------------------------------------------------------------ record policies
// How a record form is laid out, fetched and tested, and how a packet is held.
// A View locates the records of rules [0, n) either in global memory or in
// the block's shared-memory prefix (same layout in both).
struct PolClamp {
    using Rec = RecClamp;
    using Pk = Pkt;
    struct R {
        uint4 a, b;
    };
    struct View {
        const Rec *rec;
    };
    static __host__ __device__ size_t bytes_per_rule() { return sizeof(Rec); }
    static __device__ __forceinline__ View global_view(const ScanParams &p) {
        return {reinterpret_cast<const Rec *>(p.rec)};
    }
    static __device__ __forceinline__ View smem_view(unsigned char *sm, int) { return {reinterpret_cast<const Rec *>(sm)}; }
    // chunk c of the shared prefix: one bulk copy of kChunkRules records
    static __device__ __forceinline__ uint32_t stage(unsigned char *sm, int, const ScanParams &p, int c, uint64_t *bar) {
        const uint32_t bytes = kChunkRules * sizeof(Rec);
        mbar_arrive_expect_tx(bar, bytes);
        bulk_load(sm + (size_t)c * bytes, reinterpret_cast<const unsigned char *>(p.rec) + (size_t)c * bytes, bytes, bar);
        return bytes;
    }
    template <bool SMEM>
    static __device__ __forceinline__ void load4(const View &v, int k, R r[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (SMEM) r[j] = {v.rec[k + j].a, v.rec[k + j].b};
            else r[j] = {__ldg(&v.rec[k + j].a), __ldg(&v.rec[k + j].b)};
        }
    }
    static __device__ __forceinline__ Pk make(uint32_t s, uint32_t d, uint32_t sp, uint32_t dp, uint32_t pr) {
        return {s, d, ports_of(sp, dp), pr};
    }
    static __device__ __forceinline__ bool mism(const Pk &p, const R &r, uint32_t) {
        return mismatch_clamp(p, r.a, r.b) != 0u;
    }
    static __device__ __forceinline__ bool all_mismatch4(const Pk &p, const R r[4], uint32_t one) {
        return mism(p, r[0], one) & mism(p, r[1], one) & mism(p, r[2], one) & mism(p, r[3], one);
    }
    // queue entry: the packet with its batch slot above the protocol byte
    static __device__ __forceinline__ uint4 pack(const Pk &p, int slot) {
        return make_uint4(p.src, p.dst, p.ports, p.proto | ((uint32_t)slot << 8));
    }
    static __device__ __forceinline__ Pk unpack(const uint4 &e, int &slot) {
        slot = (int)(e.w >> 8);
        return {e.x, e.y, e.z, e.w & 0xFFu};
    }
};

struct PolCmp {
    using Rec = RecCmp;
    using Pk = Pkt;
    struct R {
        uint4 a, b, c;
    };
    struct View {
        const Rec *rec;
    };
    static __host__ __device__ size_t bytes_per_rule() { return sizeof(Rec); }
    static __device__ __forceinline__ View global_view(const ScanParams &p) {
        return {reinterpret_cast<const Rec *>(p.rec)};
    }
    static __device__ __forceinline__ View smem_view(unsigned char *sm, int) { return {reinterpret_cast<const Rec *>(sm)}; }
    static __device__ __forceinline__ uint32_t stage(unsigned char *sm, int, const ScanParams &p, int c, uint64_t *bar) {
        const uint32_t bytes = kChunkRules * sizeof(Rec);
        mbar_arrive_expect_tx(bar, bytes);
        bulk_load(sm + (size_t)c * bytes, reinterpret_cast<const unsigned char *>(p.rec) + (size_t)c * bytes, bytes, bar);
        return bytes;
    }
    template <bool SMEM>
    static __device__ __forceinline__ void load4(const View &v, int k, R r[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (SMEM) r[j] = {v.rec[k + j].a, v.rec[k + j].b, v.rec[k + j].c};
            else r[j] = {__ldg(&v.rec[k + j].a), __ldg(&v.rec[k + j].b), __ldg(&v.rec[k + j].c)};
        }
    }
    static __device__ __forceinline__ Pk make(uint32_t s, uint32_t d, uint32_t sp, uint32_t dp, uint32_t pr) {
        return {s, d, ports_of(sp, dp), pr};
    }
    static __device__ __forceinline__ bool mism(const Pk &p, const R &r, uint32_t) {
        return !match_cmp(p, r.a, r.b, r.c);
    }
    static __device__ __forceinline__ bool all_mismatch4(const Pk &p, const R r[4], uint32_t one) {
        return mism(p, r[0], one) & mism(p, r[1], one) & mism(p, r[2], one) & mism(p, r[3], one);
    }
    static __device__ __forceinline__ uint4 pack(const Pk &p, int slot) { return PolClamp::pack(p, slot); }
    static __device__ __forceinline__ Pk unpack(const uint4 &e, int &slot) { return PolClamp::unpack(e, slot); }
};

struct PolArith {
    using Rec = RecArith;
    using Pk = PktA;
    struct R {
        uint4 a, b;
        uint32_t w;
    };
    struct View {
        const Rec *rec;
        const uint32_t *wtop;
    };
    static __host__ __device__ size_t bytes_per_rule() { return sizeof(Rec) + sizeof(uint32_t); }
    static __device__ __forceinline__ View global_view(const ScanParams &p) {
        return {reinterpret_cast<const Rec *>(p.rec), p.wtop};
    }
    // the same records seen from record `off` on (a sub-list of the partition)
    static __device__ __forceinline__ View shifted(const View &v, int off) { return {v.rec + off, v.wtop + off}; }
    // shared layout: [n_smem records][n_smem wtop words]
    static __device__ __forceinline__ View smem_view(unsigned char *sm, int n_smem) {
        return {reinterpret_cast<const Rec *>(sm), reinterpret_cast<const uint32_t *>(sm + (size_t)n_smem * sizeof(Rec))};
    }
    static __device__ __forceinline__ uint32_t stage(unsigned char *sm, int n_smem, const ScanParams &p, int c,
                                                     uint64_t *bar) {
        const uint32_t rb = kChunkRules * sizeof(Rec), wb = kChunkRules * sizeof(uint32_t);
        mbar_arrive_expect_tx(bar, rb + wb);
        bulk_load(sm + (size_t)c * rb, reinterpret_cast<const unsigned char *>(p.rec) + (size_t)c * rb, rb, bar);
        bulk_load(sm + (size_t)n_smem * sizeof(Rec) + (size_t)c * wb,
                  reinterpret_cast<const unsigned char *>(p.wtop) + (size_t)c * wb, wb, bar);
        return rb + wb;
    }
    template <bool SMEM>
    static __device__ __forceinline__ void load4(const View &v, int k, R r[4]) {
        const uint4 w = SMEM ? *reinterpret_cast<const uint4 *>(v.wtop + k)
                             : __ldg(reinterpret_cast<const uint4 *>(v.wtop + k));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (SMEM) {
                r[j].a = v.rec[k + j].a;
                r[j].b = v.rec[k + j].b;
            } else {
                r[j].a = __ldg(&v.rec[k + j].a);
                r[j].b = __ldg(&v.rec[k + j].b);
            }
        }
        r[0].w = w.x;
        r[1].w = w.y;
        r[2].w = w.z;
        r[3].w = w.w;
    }
    static __device__ __forceinline__ Pk make(uint32_t s, uint32_t d, uint32_t sp, uint32_t dp, uint32_t pr) {
        return {s, d, sp, x_of(pr, dp)};
    }
    static __device__ __forceinline__ bool mism(const Pk &p, const R &r, uint32_t one) {
        return mismatch_arith(p, r.a, r.b, r.w, one);
    }
    static __device__ __forceinline__ bool all_mismatch4(const Pk &p, const R r[4], uint32_t one) {
        return mism(p, r[0], one) & mism(p, r[1], one) & mism(p, r[2], one) & mism(p, r[3], one);
    }
    // Bit j set exactly when rule j of the four matches. Each rule's four field
    // tests form one predicate chain as in mismatch_arith, and a predicated OR
    // records a match, so only one predicate is live and the first match is read
    // from the mask instead of testing the rules again.
    static __device__ __forceinline__ uint32_t match_mask4(const Pk &p, const R r[4], uint32_t one) {
        uint32_t ts[4], td[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ts[j] = p.sport * one + r[j].b.x;
            td[j] = p.x * r[j].b.z + r[j].b.w;
        }
        uint32_t m;
#define FW_RULE_TESTS(TS, SW, AX, AY, AZ, AW, TD, W, BIT)          \
    "setp.gt.u32 q, %" #TS ", %" #SW ";\n\t"                       \
    "lop3.or.b32 t|q, %1, %" #AX ", %" #AY ", 0x28, q;\n\t"        \
    "lop3.or.b32 t|q, %2, %" #AZ ", %" #AW ", 0x28, q;\n\t"        \
    "setp.gt.or.u32 q, %" #TD ", %" #W ", q;\n\t"                  \
    "@!q or.b32 %0, %0, " #BIT ";\n\t"
        asm("{\n\t"
            ".reg .pred q;\n\t"
            ".reg .b32 t;\n\t"
            "mov.b32 %0, 0;\n\t"
            FW_RULE_TESTS(3, 4, 5, 6, 7, 8, 9, 10, 1)
            FW_RULE_TESTS(11, 12, 13, 14, 15, 16, 17, 18, 2)
            FW_RULE_TESTS(19, 20, 21, 22, 23, 24, 25, 26, 4)
            FW_RULE_TESTS(27, 28, 29, 30, 31, 32, 33, 34, 8)
            "}"
            : "=&r"(m)
            : "r"(p.src), "r"(p.dst),
              "r"(ts[0]), "r"(r[0].b.y), "r"(r[0].a.x), "r"(r[0].a.y), "r"(r[0].a.z), "r"(r[0].a.w), "r"(td[0]), "r"(r[0].w),
              "r"(ts[1]), "r"(r[1].b.y), "r"(r[1].a.x), "r"(r[1].a.y), "r"(r[1].a.z), "r"(r[1].a.w), "r"(td[1]), "r"(r[1].w),
              "r"(ts[2]), "r"(r[2].b.y), "r"(r[2].a.x), "r"(r[2].a.y), "r"(r[2].a.z), "r"(r[2].a.w), "r"(td[2]), "r"(r[2].w),
              "r"(ts[3]), "r"(r[3].b.y), "r"(r[3].a.x), "r"(r[3].a.y), "r"(r[3].a.z), "r"(r[3].a.w), "r"(td[3]), "r"(r[3].w));
#undef FW_RULE_TESTS
        return m;
    }
    // queue entry: the batch slot above the 16-bit source port
    static __device__ __forceinline__ uint4 pack(const Pk &p, int slot) {
        return make_uint4(p.src, p.dst, p.sport | ((uint32_t)slot << 16), p.x);
    }
    static __device__ __forceinline__ Pk unpack(const uint4 &e, int &slot) {
        slot = (int)(e.z >> 16);
        return {e.x, e.y, e.z & 0xFFFFu, e.w};
    }
};

// Range form: the arithmetic-form layout with every field a range test.
struct PolRange : PolArith {
    static __device__ __forceinline__ bool mism(const Pk &p, const R &r, uint32_t one) {
        return mismatch_range_c(p, r.a, r.b, r.w, one);
    }
    static __device__ __forceinline__ bool all_mismatch4(const Pk &p, const R r[4], uint32_t one) {
        uint32_t t[16], w[16];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            t[4 * j + 0] = p.src * one + r[j].a.x;
            w[4 * j + 0] = r[j].a.y;
            t[4 * j + 1] = p.dst * one + r[j].a.z;
            w[4 * j + 1] = r[j].a.w;
            t[4 * j + 2] = p.sport * one + r[j].b.x;
            w[4 * j + 2] = r[j].b.y;
            t[4 * j + 3] = p.x * r[j].b.z + r[j].b.w;
            w[4 * j + 3] = r[j].w;
        }
        return all_mismatch4_range(t, w) != 0u;
    }
};

// ------------------------------------------------------------ packet loads
template <class Pol, bool VEC>
__device__ __forceinline__ void load_quad(const HdrPtrs &h, int64_t n, int64_t q, typename Pol::Pk pk[4],
                                          int &cnt) {
    const int64_t base = q * 4;
    if (VEC && base + 3 < n) {
        uint4 s = __ldcs(reinterpret_cast<const uint4 *>(h.src) + q);
        uint4 d = __ldcs(reinterpret_cast<const uint4 *>(h.dst) + q);
        uint2 sp = __ldcs(reinterpret_cast<const uint2 *>(h.sport) + q);
        uint2 dp = __ldcs(reinterpret_cast<const uint2 *>(h.dport) + q);
        uint32_t pr = __ldcs(reinterpret_cast<const unsigned int *>(h.proto) + q);
        pk[0] = Pol::make(s.x, d.x, sp.x & 0xFFFFu, dp.x & 0xFFFFu, pr & 0xFFu);
        pk[1] = Pol::make(s.y, d.y, sp.x >> 16, dp.x >> 16, (pr >> 8) & 0xFFu);
        pk[2] = Pol::make(s.z, d.z, sp.y & 0xFFFFu, dp.y & 0xFFFFu, (pr >> 16) & 0xFFu);
        pk[3] = Pol::make(s.w, d.w, sp.y >> 16, dp.y >> 16, pr >> 24);
        cnt = 4;
    } else {
        cnt = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t i = base + j;
            if (i < n) {
                pk[j] = Pol::make(h.src[i], h.dst[i], h.sport[i], h.dport[i], h.proto[i]);
                cnt = j + 1;
            } else {
                pk[j] = Pol::make(0, 0, 0, 0, 0);
            }
        }
    }
}

template <bool VEC>
__device__ __forceinline__ void store_quad(const ScanParams &p, int64_t q, const int idx[4], int cnt) {
    const int64_t base = q * 4;
    uint32_t a[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = idx[j] >= 0 ? __ldg(p.action + idx[j]) : (uint32_t)FW_DROP;
    if (VEC && cnt == 4) {
        __stcs(reinterpret_cast<int4 *>(p.out_idx) + q, make_int4(idx[0], idx[1], idx[2], idx[3]));
        __stcs(reinterpret_cast<unsigned int *>(p.out_act) + q, a[0] | (a[1] << 8) | (a[2] << 16) | (a[3] << 24));
    } else {
        for (int j = 0; j < cnt; ++j) {
            p.out_idx[base + j] = idx[j];
            p.out_act[base + j] = (uint8_t)a[j];
        }
    }
}

// ------------------------------------------------------------ rule scans
// Rules k..k+3 against one packet: k + (first of the four that matches), or -1.
template <class Pol, bool SMEM>
__device__ __forceinline__ int scan_block4(const typename Pol::Pk &pk, const typename Pol::View &v, int k,
                                           uint32_t one) {
    typename Pol::R r[4];
    Pol::template load4<SMEM>(v, k, r);
    if (Pol::all_mismatch4(pk, r, one)) return -1;
    // once per decided packet: which of the four matched first
    return k + (!Pol::mism(pk, r[0], one) ? 0 : !Pol::mism(pk, r[1], one) ? 1 : !Pol::mism(pk, r[2], one) ? 2 : 3);
}

// First index in [k0, k1) whose rule matches, or -1 (k0, k1 multiples of 4).
// Rules below n_smem come from the block's shared-memory prefix (already
// resident: see stage_rules), the rest from global memory.
template <class Pol>
__device__ __forceinline__ int scan_range(const typename Pol::Pk &pk, int k0, int k1, const typename Pol::View &sv,
                                          int n_smem, const typename Pol::View &gv, uint32_t one) {
    int k = k0;
    const int lim = min(k1, n_smem);
    for (; k < lim; k += 4) {
        const int r = scan_block4<Pol, true>(pk, sv, k, one);
        if (r >= 0) return r;
    }
    for (; k < k1; k += 4) {
        const int r = scan_block4<Pol, false>(pk, gv, k, one);
        if (r >= 0) return r;
    }
    return -1;
}

// Two packets against the same rules: each rule record is loaded once for
// both, and the two packets' tests are independent chains the scheduler can
// overlap. ra / rb as scan_range for packets a / b (a packet that is not
// valid is not scanned and returns -1). The loop runs until both are decided.
template <class Pol>
__device__ __forceinline__ void scan_range2(const typename Pol::Pk &a, const typename Pol::Pk &b, bool va, bool vb,
                                            int k0, int k1, const typename Pol::View &sv, int n_smem,
                                            const typename Pol::View &gv, uint32_t one, int &ra, int &rb) {
    static_assert(std::is_same<Pol, PolArith>::value, "two-packet scan: arithmetic record form only");
    ra = -1;
    rb = -1;
    bool da = !va, db = !vb;
    int k = k0;
    const int lim = min(k1, n_smem);
    for (; k < lim && !(da && db); k += 4) {
        typename Pol::R r[4];
        Pol::template load4<true>(sv, k, r);
        const uint32_t ma = Pol::match_mask4(a, r, one), mb = Pol::match_mask4(b, r, one);
        if (!da && ma) {
            ra = k + __ffs(ma) - 1;
            da = true;
        }
        if (!db && mb) {
            rb = k + __ffs(mb) - 1;
            db = true;
        }
    }
    for (; k < k1 && !(da && db); k += 4) {
        typename Pol::R r[4];
        Pol::template load4<false>(gv, k, r);
        const uint32_t ma = Pol::match_mask4(a, r, one), mb = Pol::match_mask4(b, r, one);
        if (!da && ma) {
            ra = k + __ffs(ma) - 1;
            da = true;
        }
        if (!db && mb) {
            rb = k + __ffs(mb) - 1;
            db = true;
        }
    }
}

// Shared-memory rule prefix: one mbarrier per 256-rule chunk, the chunks
// brought in by 1-D TMA bulk copies issued by thread 0, then every thread
// waits (bounded) until all chunks have landed. A persistent block does this
// once and then serves millions of packets from the prefix. Returns false if
// a wait gave up (the status word is set; the caller must not use the prefix).
template <class Pol>
__device__ __forceinline__ bool stage_rules(unsigned char *smem, const ScanParams &p) {
    const int n_chunks = p.n_smem / kChunkRules;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)p.n_smem * Pol::bytes_per_rule());
    if (threadIdx.x == 0) {
        for (int c = 0; c < n_chunks; ++c) mbar_init(&bars[c], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int c = 0; c < n_chunks; ++c) Pol::stage(smem, p.n_smem, p, c, &bars[c]);
    bool ok = true;
    for (int c = 0; c < n_chunks; ++c) ok = mbar_wait_bounded(&bars[c], 0, p.status) && ok;
    return __syncthreads_and(ok) != 0;
}

// After a failed stage_rules: before the block exits, give copies that may
// still be in flight into its shared memory a second bounded wait.
template <class Pol>
__device__ __forceinline__ void drain_rules(unsigned char *smem, const ScanParams &p) {
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)p.n_smem * Pol::bytes_per_rule());
    if (threadIdx.x == 0)
        for (int c = 0; c < p.n_smem / kChunkRules; ++c) mbar_wait_bounded(&bars[c], 0, p.status);
}

// Protocol bytes of quad q (packets 4q..4q+3) packed little-endian into pr4;
// nv = how many of the four exist (0 when !in_batch).
template <bool VEC>
__device__ __forceinline__ void load_protos(const HdrPtrs &h, int64_t n, int64_t q, bool in_batch, uint32_t &pr4,
                                            int &nv) {
    pr4 = 0;
    nv = 0;
    if (!in_batch) return;
    const int64_t b = q * 4;
    if (VEC && b + 3 < n) {
        pr4 = __ldg(reinterpret_cast<const unsigned int *>(h.proto) + q);
        nv = 4;
        return;
    }
    for (int j = 0; j < 4 && b + j < n; ++j) {
        pr4 |= (uint32_t)h.proto[b + j] << (8 * j);
        nv = j + 1;
    }
}

// Partition classes of quad q (packets 4q..4q+3) for a count pass: the protocol
// bytes, plus the keyed address words when the partition has an address key;
// nv = how many of the four exist.
template <bool VEC, class T>
__device__ __forceinline__ void load_classes4(const T &t, int64_t q, uint32_t cls[4], int &nv) {
    uint32_t pr4;
    load_protos<VEC>(t.h, t.n, q, true, pr4, nv);
    uint32_t a[4] = {0, 0, 0, 0};
    if (t.key_field != 0) {
        const uint32_t *arr = t.key_field == 1 ? t.h.src : t.h.dst;
        const int64_t b = q * 4;
        if (VEC && nv == 4) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(arr) + q);
            a[0] = v.x;
            a[1] = v.y;
            a[2] = v.z;
            a[3] = v.w;
        } else {
            for (int j = 0; j < nv; ++j) a[j] = arr[b + j];
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
        cls[j] = part_class(t.class_of[(pr4 >> (8 * j)) & 0xFFu], t.key_field, t.key_bits, a[j], a[j]);
}

// Protocol of a packet held in a policy's packet form (the partition key).
template <class Pol>
__device__ __forceinline__ uint32_t pkt_proto(const typename Pol::Pk &p);
template <>
__device__ __forceinline__ uint32_t pkt_proto<PolArith>(const PolArith::Pk &p) { return p.x >> 17; }
template <>
__device__ __forceinline__ uint32_t pkt_proto<PolRange>(const PolRange::Pk &p) { return p.x >> 17; }
template <>
__device__ __forceinline__ uint32_t pkt_proto<PolClamp>(const PolClamp::Pk &p) { return p.proto; }
template <>
__device__ __forceinline__ uint32_t pkt_proto<PolCmp>(const PolCmp::Pk &p) { return p.proto; }

// View of a sub-list that starts `off` records into the stored array (arithmetic form only).
template <class Pol>
__device__ __forceinline__ typename Pol::View shifted_view(const typename Pol::View &v, int off) {
    return PolArith::shifted(v, off);
}


// ------------------------------------------------------------ one warp batch
// What a warp needs to classify a batch: the headers, the rule records (the
// shared prefix and the global array, or the protocol partition), and where
// the verdicts go.
template <class Pol>
struct BatchTarget {
    HdrPtrs h;
    int64_t n;                        // packets in the whole array
    typename Pol::View sv, gv;        // shared-memory prefix / global records
    int n_smem;                       // records resident in the shared prefix
    int n_scan;                       // records of the whole list (unpartitioned)
    int n_classes;                    // partition: classes, address key, sub-list offsets and
    int key_field, key_bits;          //   lengths, protocol -> protocol class table, original
    const int32_t *class_off;         //   rule index
    const int32_t *class_len;
    const uint8_t *class_of;
    const int32_t *orig;
    const uint32_t *verdict;          // partition: original index | action << 31 per record
    const uint8_t *action;
    int32_t *out_idx;
    uint8_t *out_act;
    int seg0;                         // first rule segment; later segments double
    uint32_t one;
};

// Classify packets [base, base + cnt) with one warp. The batch goes into the
// warp's shared queue Q (PART: counting-sorted by protocol class, one region
// per class; wc = 2 * kMaxClasses ints of per-warp counters). Each region is
// scanned segment by segment over its rule list; after each group of 32
// queue entries, packets decided in the segment write their verdicts and the
// undecided ones are packed to the front of the region (ballot + popc), so
// the next segment runs on dense groups of still-undecided packets instead of
// lanes idling behind the slowest packet of a warp.
template <class Pol, bool VEC, bool PART>
__device__ __forceinline__ void run_batch(const BatchTarget<Pol> &t, int64_t base, int cnt, uint4 *Q, int *wc,
                                          int lane) {
    int n_groups = 1;
    if constexpr (PART) {
        // count (shared atomics, one per packet), exclusive prefix, scatter
        n_groups = t.n_classes;
        if (lane < 2 * kMaxClasses) wc[lane] = 0;
        __syncwarp();
        for (int qq = lane; qq * 4 < cnt; qq += 32) {
            uint32_t cls[4];
            int nv;
            load_classes4<VEC>(t, base / 4 + qq, cls, nv);
            for (int j = 0; j < nv; ++j) atomicAdd(&wc[cls[j]], 1);
        }
        __syncwarp();
        if (lane == 0) {
            int acc = 0;
            for (int c = 0; c < t.n_classes; ++c) {
                wc[kMaxClasses + c] = acc;  // region start; advanced by the scatter below
                acc += wc[c];
            }
        }
        __syncwarp();
        for (int qq = lane; qq * 4 < cnt; qq += 32) {
            typename Pol::Pk pk[4];
            int nv;
            load_quad<Pol, VEC>(t.h, t.n, base / 4 + qq, pk, nv);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j >= nv) continue;
                const uint32_t c = part_class(t.class_of[pkt_proto<Pol>(pk[j]) & 0xFFu], t.key_field, t.key_bits,
                                              pk[j].src, pk[j].dst);
                const int pos = atomicAdd(&wc[kMaxClasses + c], 1);
                Q[pos] = Pol::pack(pk[j], qq * 4 + j);
            }
        }
    } else {
        for (int qq = lane; qq * 4 < cnt; qq += 32) {
            typename Pol::Pk pk[4];
            int c;
            load_quad<Pol, VEC>(t.h, t.n, base / 4 + qq, pk, c);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (j < c) Q[qq * 4 + j] = Pol::pack(pk[j], qq * 4 + j);
        }
    }
    __syncwarp();
    for (int g = 0; g < n_groups; ++g) {
        int m = cnt, R = 0, off = 0, len = t.n_scan;
        typename Pol::View svg = t.sv, gvg = t.gv;
        if constexpr (PART) {
            m = wc[g];
            R = wc[kMaxClasses + g] - m;  // region of class g (the scatter left its pointer at the end)
            off = t.class_off[g];
            len = t.class_len[g];
            svg = shifted_view<Pol>(t.sv, off);
            gvg = shifted_view<Pol>(t.gv, off);
        }
        const int n_smem_g = max(0, t.n_smem - off);
        int s0 = 0, s1 = t.seg0;
        while (m > 0) {
            s1 = min(s1, len);
            const bool last = s1 >= len;
            int w = 0;
            for (int g0 = 0; g0 < m; g0 += 32) {
                const int i = g0 + lane;
                const bool valid = i < m;
                const uint4 e = valid ? Q[R + i] : make_uint4(0, 0, 0, 0);
                __syncwarp();
                int slot;
                const typename Pol::Pk pk = Pol::unpack(e, slot);
                int r = -1;
                if (valid && s0 < s1) r = scan_range<Pol>(pk, s0, s1, svg, n_smem_g, gvg, t.one);
                const bool keep = valid && r == -1 && !last;
                if (valid && !keep) {
                    int v = r;
                    if constexpr (PART) v = r >= 0 ? __ldg(t.orig + off + r) : -1;
                    v = v >= 0 ? v : -1;
                    t.out_idx[base + slot] = v;
                    t.out_act[base + slot] = v >= 0 ? __ldg(t.action + v) : (uint8_t)FW_DROP;
                }
                const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
                if (keep) Q[R + w + __popc(bal & ((1u << lane) - 1u))] = e;
                w += __popc(bal);
                __syncwarp();
            }
            m = w;
            s0 = s1;
            s1 = s1 * 2;
        }
    }
    __syncwarp();
}

// Queue index of sorted position `pos` in the two-packets-per-lane layout: lane l
// of a 64-entry group holds sorted entries 2l and 2l+1, stored at l and 32 + l,
// so each of the group's two loads reads 32 consecutive 16-byte entries.
__device__ __forceinline__ int pair_slot(int pos) { return (pos & ~63) + ((pos & 1) << 5) + ((pos >> 1) & 31); }

// Slot value of a queue entry that holds no packet to scan: the pad that makes a
// class region even, or a packet decided in the last segment. Real slots are
// below the queue capacity, which shared memory bounds far below 0xFFFF.
constexpr uint32_t kNoSlot = 0xFFFFu;

// Per-lane class counters: 16-bit fields, four classes to a 64-bit word.
struct ClassCounts {
    uint64_t w[kMaxClasses / 4];
};
static_assert(kMaxClasses == 8, "ClassCounts selects between two words");
__device__ __forceinline__ uint32_t class_field(const ClassCounts &k, uint32_t c) {
    return (uint32_t)((c < 4 ? k.w[0] : k.w[1]) >> (16 * (c & 3))) & 0xFFFFu;
}
__device__ __forceinline__ void class_bump(ClassCounts &k, uint32_t c) {
    const uint64_t inc = 1ull << (16 * (c & 3));
    if (c < 4) k.w[0] += inc;
    else k.w[1] += inc;
}

// Queue entries of the two-packet scan carry their class in bits 28-30 of the
// fourth word, above the 25 bits of (protocol << 17 | dport).
constexpr uint32_t kXMask = 0x01FFFFFFu;
__device__ __forceinline__ uint32_t entry_class(const uint4 &e) { return e.w >> 28; }

// After the re-sort (cur[c] = start + count): one pad entry behind every
// odd-sized region.
__device__ __forceinline__ void write_pads(int n_classes, const int *cnt, const int *cur, uint4 *Q, int lane) {
    if (lane < n_classes && (cnt[lane] & 1)) Q[pair_slot(cur[lane])] = make_uint4(0, 0, kNoSlot << 16, 0);
    __syncwarp();
}

// Lane 0 sets cur[c] to the start of class c's region, each region padded to an
// even count; returns the padded total (every lane).
__device__ __forceinline__ int even_region_starts(int n_classes, const int *cnt, int *cur, int lane) {
    int acc = 0;
    for (int c = 0; c < n_classes; ++c) {
        if (lane == 0) cur[c] = acc;
        acc += (cnt[c] + 1) & ~1;
    }
    __syncwarp();
    return acc;
}

// run_batch with two packets per lane (partitioned arithmetic form). The batch
// is sorted by protocol class, every class region padded to an even count, so
// the two entries a lane holds always share a class: one rule load from their
// sub-list feeds both tests. A 64-entry group may span classes; each lane
// follows its own class's sub-list (the loads of a group then have as many
// distinct addresses as it has classes). The sort needs no atomics: each lane
// counts its own packets per class in registers, one warp-wide exclusive scan
// of those counters gives every lane its place in each region, and the lane
// writes its packets there. The queue holds cnt plus at most n_classes pads.
// After a segment that is not the last for every class, the undecided packets
// are re-sorted by class, padded again, in place: regions only shrink, so a
// packet's new position never lies past the group being read.
template <class Pol, bool VEC>
__device__ __forceinline__ void run_batch_pairs(const BatchTarget<Pol> &t, int64_t base, int cnt, uint4 *Q, int *wc,
                                                int lane) {
    int *cnt_c = wc, *cur_c = wc + kMaxClasses;
    const int nc = t.n_classes;
    ClassCounts own{};
    for (int qq = lane; qq * 4 < cnt; qq += 32) {
        uint32_t cls[4];
        int nv;
        load_classes4<VEC>(t, base / 4 + qq, cls, nv);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < nv) class_bump(own, cls[j]);
    }
    ClassCounts ex = own, tot;  // inclusive scan over lanes, then exclusive
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
        for (int i = 0; i < kMaxClasses / 4; ++i) {
            const uint64_t a = __shfl_up_sync(0xFFFFFFFFu, ex.w[i], d);
            if (lane >= d) ex.w[i] += a;
        }
    }
#pragma unroll
    for (int i = 0; i < kMaxClasses / 4; ++i) {
        tot.w[i] = __shfl_sync(0xFFFFFFFFu, ex.w[i], 31);
        ex.w[i] -= own.w[i];
    }
    int m = 0;
    for (int c = 0; c < nc; ++c) {
        const int tc = (int)class_field(tot, (uint32_t)c);
        if (lane == 0) {
            cur_c[c] = m;
            cnt_c[c] = tc;
        }
        m += (tc + 1) & ~1;
    }
    __syncwarp();
    for (int qq = lane; qq * 4 < cnt; qq += 32) {
        typename Pol::Pk pk[4];
        int nv;
        load_quad<Pol, VEC>(t.h, t.n, base / 4 + qq, pk, nv);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j >= nv) continue;
            const uint32_t c = part_class(t.class_of[pkt_proto<Pol>(pk[j]) & 0xFFu], t.key_field, t.key_bits,
                                          pk[j].src, pk[j].dst);
            const int pos = cur_c[c] + (int)class_field(ex, c);
            class_bump(ex, c);
            uint4 e = Pol::pack(pk[j], qq * 4 + j);
            e.w |= c << 28;
            Q[pair_slot(pos)] = e;
        }
    }
    if (lane < nc && (cnt_c[lane] & 1)) Q[pair_slot(cur_c[lane] + cnt_c[lane])] = make_uint4(0, 0, kNoSlot << 16, 0);
    __syncwarp();
    int max_len = 0;
    for (int c = 0; c < nc; ++c) max_len = max(max_len, t.class_len[c]);
    int s0 = 0, s1 = t.seg0;
    while (m > 0) {
        const bool final_seg = s1 >= max_len;  // every class's sub-list ends in this segment
        if (!final_seg) {
            if (lane < kMaxClasses) cnt_c[lane] = 0;
            __syncwarp();
        }
        for (int g0 = 0; g0 < m; g0 += 64) {
            const bool in = g0 + 2 * lane < m;  // m is even: both entries of the lane or neither
            uint4 e0 = in ? Q[g0 + lane] : make_uint4(0, 0, kNoSlot << 16, 0);
            uint4 e1 = in ? Q[g0 + 32 + lane] : make_uint4(0, 0, kNoSlot << 16, 0);
            const uint32_t cls = entry_class(e0);  // a pad is only ever second; both share the class
            e0.w &= kXMask;
            e1.w &= kXMask;
            int slot0, slot1;
            const typename Pol::Pk a = Pol::unpack(e0, slot0), b = Pol::unpack(e1, slot1);
            const bool v0 = slot0 != (int)kNoSlot, v1 = slot1 != (int)kNoSlot;
            const int off = v0 ? t.class_off[cls] : 0, len = v0 ? t.class_len[cls] : 0;
            const int k1 = min(s1, len);
            const bool last = s1 >= len;
            int r0 = -1, r1 = -1;
            if (v0 && s0 < k1)
                scan_range2<Pol>(a, b, v0, v1, s0, k1, shifted_view<Pol>(t.sv, off), max(0, t.n_smem - off),
                                 shifted_view<Pol>(t.gv, off), t.one, r0, r1);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const bool valid = u ? v1 : v0;
                const int r = u ? r1 : r0, slot = u ? slot1 : slot0;
                const bool decided = valid && (r >= 0 || last);
                if (decided) {
                    const uint32_t w = r >= 0 ? __ldg(t.verdict + off + r) : 0xFFFFFFFFu;
                    t.out_idx[base + slot] = r >= 0 ? (int32_t)(w & 0x7FFFFFFFu) : -1;
                    t.out_act[base + slot] = r >= 0 ? (uint8_t)(w >> 31) : (uint8_t)FW_DROP;
                }
                if (!final_seg) {
                    if (valid && !decided) atomicAdd(&cnt_c[cls], 1);
                    else if (decided) Q[g0 + 32 * u + lane].z = kNoSlot << 16;
                }
            }
        }
        if (final_seg) break;
        __syncwarp();
        const int m_old = m;
        m = even_region_starts(nc, cnt_c, cur_c, lane);
        for (int g0 = 0; g0 < m_old; g0 += 64) {
            const bool in = g0 + 2 * lane < m_old;
            const uint4 e0 = in ? Q[g0 + lane] : make_uint4(0, 0, kNoSlot << 16, 0);
            const uint4 e1 = in ? Q[g0 + 32 + lane] : make_uint4(0, 0, kNoSlot << 16, 0);
            __syncwarp();
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const uint4 e = u ? e1 : e0;
                if ((e.z >> 16) != kNoSlot) {
                    const int pos = atomicAdd(&cur_c[entry_class(e)], 1);
                    Q[pair_slot(pos)] = e;
                }
            }
            __syncwarp();
        }
        write_pads(nc, cnt_c, cur_c, Q, lane);
        s0 = s1;
        s1 = s1 * 2;
    }
    __syncwarp();
}

}  // namespace fwk
