// Rule-set construction: validation, canonicalisation and upload.
//
// The rule model is the paper's 5-tuple with wildcard fields (Sec. IV): an
// address is matched under a prefix mask, ports under inclusive ranges, the
// protocol exactly or not at all. Canonicalisation turns each rule into the
// two device record forms described in fw_internal.cuh and records the first
// catch-all rule (all five fields wildcards): under first match (Sec. I) no
// packet is ever decided by a rule after it, so scans stop there.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fw_alloc.h"
#include "fw_internal.cuh"

namespace fwk {

static thread_local int g_last_status = FW_OK;

// Allocation-failure injection (fw_selftest_fail_alloc): allocations left
// before the one that fails, or -1 when disarmed.
static std::atomic<int64_t> g_fail_after{-1};

bool take_injected_alloc_failure() {
    int64_t k = g_fail_after.load(std::memory_order_relaxed);
    while (k >= 0) {
        if (g_fail_after.compare_exchange_weak(k, k == 0 ? -1 : k - 1, std::memory_order_relaxed))
            return k == 0;
    }
    return false;
}

int set_status(int s) {
    if (s != FW_OK) g_last_status = s;
    return s;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return FW_OK;
    if (e == cudaErrorMemoryAllocation) return FW_ENOMEM;
    return FW_ECUDA;
}

int check_device(const fw_ruleset *rs) {
    int dev = -1;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e);
    }
    return dev == rs->device ? FW_OK : FW_EINVAL;
}

uint32_t prefix_mask(unsigned prefix) {
    return prefix == 0 ? 0u : (0xFFFFFFFFu << (32u - prefix));
}

bool is_catch_all(const fw_rule &r) {
    return r.src_prefix == 0 && r.dst_prefix == 0 && r.sport_lo == 0 && r.sport_hi == 0xFFFF && r.dport_lo == 0 &&
           r.dport_hi == 0xFFFF && r.proto_any != 0;
}

int validate_rule(const fw_rule &r) {
    if (r.src_prefix > 32 || r.dst_prefix > 32) return FW_EINVAL;
    if (r.sport_lo > r.sport_hi || r.dport_lo > r.dport_hi) return FW_EINVAL;
    if (r.action != FW_DROP && r.action != FW_ACCEPT) return FW_EINVAL;
    if (r.reserved[0] | r.reserved[1] | r.reserved[2]) return FW_EINVAL;
    return FW_OK;
}

static void canon_arith(const fw_rule &r, RecArith *q, uint32_t *wt) {
    uint32_t sm = prefix_mask(r.src_prefix), dm = prefix_mask(r.dst_prefix);
    q->a = make_uint4(r.src_addr & sm, sm, r.dst_addr & dm, dm);
    const uint32_t dw = uint32_t(r.dport_hi) - r.dport_lo;
    uint32_t mul, add, wtop;
    if (r.proto_any) {
        mul = 1u << 15;
        add = 0u - (uint32_t(r.dport_lo) << 15);
        wtop = dw << 15;
    } else {
        mul = 1u;
        add = 0u - ((uint32_t(r.proto) << 17) | r.dport_lo);
        wtop = dw;
    }
    q->b = make_uint4(0u - uint32_t(r.sport_lo), uint32_t(r.sport_hi) - r.sport_lo, mul, add);
    *wt = wtop;
}

static void canon_range(const fw_rule &r, RecRange *q, uint32_t *wt) {
    canon_arith(r, q, wt);  // ports and protocol as in the arithmetic form
    uint32_t sm = prefix_mask(r.src_prefix), dm = prefix_mask(r.dst_prefix);
    const uint32_t slo = r.src_addr & sm, dlo = r.dst_addr & dm;
    q->a = make_uint4(0u - slo, ~sm, 0u - dlo, ~dm);
}

static void never_match_arith(RecArith *q, uint32_t *wt) {
    q->a = make_uint4(0, 0, 0, 0);
    // exact protocol 0x100: no 8-bit protocol reaches the window
    q->b = make_uint4(0u, 0xFFFFFFFFu, 1u, 0u - (kNeverProto << 17));
    *wt = 0u;
}

static void canon(const fw_rule &r, RecClamp *c, RecCmp *m) {
    uint32_t sm = prefix_mask(r.src_prefix), dm = prefix_mask(r.dst_prefix);
    uint32_t pm = r.proto_any ? 0u : 0xFFu;
    uint32_t pv = r.proto_any ? 0u : r.proto;
    c->a = make_uint4(r.src_addr & sm, sm, r.dst_addr & dm, dm);
    c->b = make_uint4((uint32_t(r.sport_lo) << 16) | r.dport_lo, (uint32_t(r.sport_hi) << 16) | r.dport_hi, pv, pm);
    m->a = c->a;
    m->b = make_uint4(r.sport_lo, uint32_t(r.sport_hi) - r.sport_lo, r.dport_lo, uint32_t(r.dport_hi) - r.dport_lo);
    m->c = make_uint4(pv, pm, 0u, 0u);
}

static void never_match(RecClamp *c, RecCmp *m) {
    c->a = make_uint4(0, 0, 0, 0);
    c->b = make_uint4(0, 0xFFFFFFFFu, kNeverProto, 0xFFFFFFFFu);
    m->a = c->a;
    m->b = make_uint4(0, 0xFFFFFFFFu, 0, 0xFFFFFFFFu);
    m->c = make_uint4(kNeverProto, 0xFFFFFFFFu, 0, 0);
}

void protocol_classes(const fw_rule *rules, int64_t n, std::vector<uint8_t> &class_of,
                      std::vector<std::vector<int64_t>> &lists) {
    std::vector<int64_t> cnt(256, 0);
    for (int64_t k = 0; k < n; ++k)
        if (!rules[k].proto_any) cnt[rules[k].proto]++;
    std::vector<int> order;
    for (int p = 0; p < 256; ++p)
        if (cnt[p] > 0) order.push_back(p);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cnt[a] > cnt[b]; });
    if ((int)order.size() > kMaxProtoClasses - 1) order.resize(kMaxProtoClasses - 1);
    const int n_classes = (int)order.size() + 1;
    class_of.assign(256, (uint8_t)(n_classes - 1));
    for (size_t c = 0; c < order.size(); ++c) class_of[order[c]] = (uint8_t)c;
    lists.assign(n_classes, std::vector<int64_t>());
    for (int64_t k = 0; k < n; ++k) {
        const fw_rule &r = rules[k];
        for (int c = 0; c < n_classes; ++c) {
            const bool other = c == n_classes - 1;
            if (r.proto_any || (!other && r.proto == order[c]) || (other && class_of[r.proto] == c))
                lists[c].push_back(k);
        }
    }
}

void pack_sublists(const std::vector<std::vector<int64_t>> &lists, int32_t *class_off, int32_t *class_len) {
    int64_t off = 0;
    for (int c = 0; c < kMaxClasses; ++c) {
        const int64_t len = c < (int)lists.size() ? (int64_t)(lists[c].size() + 3) / 4 * 4 : 0;
        class_off[c] = (int32_t)off;
        class_len[c] = (int32_t)len;
        off += len;
    }
}

void partition_lists(const fw_rule *rules, int64_t n, int64_t granule, std::vector<uint8_t> &class_of,
                     std::vector<std::vector<int64_t>> &lists, int &key_field, int &key_bits) {
    std::vector<std::vector<int64_t>> plists;
    protocol_classes(rules, n, class_of, plists);
    const int np = (int)plists.size();
    auto covers = [&](const fw_rule &r, int field, int bits, uint32_t k) {
        const unsigned len = field == 1 ? r.src_prefix : r.dst_prefix;
        const uint32_t a = field == 1 ? r.src_addr : r.dst_addr;
        if (len == 0) return true;
        if (len >= (unsigned)bits) return (a >> (32 - bits)) == k;
        return (k >> (bits - len)) == (a >> (32 - len));
    };
    auto sublists = [&](int field, int bits) {
        std::vector<std::vector<int64_t>> out((size_t)np << bits);
        for (int p = 0; p < np; ++p)
            for (uint32_t k = 0; k < (1u << bits); ++k)
                for (int64_t r : plists[p])
                    if (bits == 0 || covers(rules[r], field, bits, k)) out[((size_t)p << bits) | k].push_back(r);
        return out;
    };
    auto cost = [&](size_t len) {
        return granule <= 1 ? (double)len : (double)std::max<int64_t>(1, ((int64_t)len + granule - 1) / granule);
    };
    int best_field = 0, best_bits = 0;
    double best = 0;
    for (const auto &L : plists) best += cost(L.size());
    best /= np;
    for (int field = 1; field <= 2; ++field)
        for (int bits = 1; bits <= 3 && (np << bits) <= kMaxClasses; ++bits) {
            const auto L = sublists(field, bits);
            double mean = 0;
            for (const auto &l : L) mean += cost(l.size());
            mean /= (double)L.size();
            if (mean < best) {
                best = mean;
                best_field = field;
                best_bits = bits;
            }
        }
    lists = sublists(best_field, best_bits);
    key_field = best_field;
    key_bits = best_bits;
}

}  // namespace fwk

using namespace fwk;

extern "C" int fw_ruleset_create_ex(const fw_rule *rules, int64_t n, fw_ruleset **out) {
    if (out == nullptr) return set_status(FW_EINVAL);
    *out = nullptr;
    if (n < 0 || (n > 0 && rules == nullptr) || n > (int64_t(1) << 30)) return set_status(FW_EINVAL);
    int64_t first_ca = -1;
    for (int64_t k = 0; k < n; ++k) {
        int s = validate_rule(rules[k]);
        if (s != FW_OK) return set_status(s);
        if (first_ca < 0 && is_catch_all(rules[k])) first_ca = k;
    }
    fw_ruleset *rs = new (std::nothrow) fw_ruleset();
    if (rs == nullptr) return set_status(FW_ENOMEM);
    rs->n = n;
    rs->first_catch_all = first_ca;
    rs->n_eff = first_ca >= 0 ? first_ca + 1 : n;
    rs->n_pad = ((rs->n_eff + kChunkRules - 1) / kChunkRules) * kChunkRules;
    if (rs->n_pad == 0) rs->n_pad = kChunkRules;
    cudaGetDevice(&rs->device);

    std::vector<RecClamp> hc(rs->n_pad);
    std::vector<RecCmp> hm(rs->n_pad);
    std::vector<RecArith> hq(rs->n_pad), part_rec;
    std::vector<uint32_t> part_wtop;
    std::vector<int32_t> part_orig;
    std::vector<uint32_t> part_verdict;
    std::vector<uint8_t> part_class_of;
    std::vector<std::vector<int64_t>> part_lists;
    std::vector<uint32_t> hw(rs->n_pad);
    std::vector<RecRange> hr(rs->n_pad);
    std::vector<uint32_t> hrw(rs->n_pad);
    std::vector<uint8_t> ha(rs->n_pad, FW_DROP);
    for (int64_t k = 0; k < rs->n_pad; ++k) {
        if (k < rs->n_eff) {
            canon(rules[k], &hc[k], &hm[k]);
            canon_arith(rules[k], &hq[k], &hw[k]);
            canon_range(rules[k], &hr[k], &hrw[k]);
            ha[k] = rules[k].action;
        } else {
            never_match(&hc[k], &hm[k]);
            never_match_arith(&hq[k], &hw[k]);
            never_match_arith(&hr[k], &hrw[k]);
            hr[k].a = make_uint4(0u, 0xFFFFFFFFu, 0u, 0xFFFFFFFFu);
        }
    }
    // Partition into per-class sub-lists (protocol class and address key; the
    // key is chosen by partition_lists), packed 4-aligned, one after another.
    {
        std::vector<uint8_t> class_of;
        std::vector<std::vector<int64_t>> lists;
        int key_field = 0, key_bits = 0;
        partition_lists(rules, rs->n_eff, 1, class_of, lists, key_field, key_bits);
        rs->key_field = key_field;
        rs->key_bits = key_bits;
        rs->n_classes = (int)lists.size();
        pack_sublists(lists, rs->class_off, rs->class_len);
        const int64_t off = rs->class_off[kMaxClasses - 1] + rs->class_len[kMaxClasses - 1];
        rs->part_pad = std::max<int64_t>(kChunkRules, (off + kChunkRules - 1) / kChunkRules * kChunkRules);
        part_rec.resize(rs->part_pad);
        part_wtop.resize(rs->part_pad);
        part_orig.assign(rs->part_pad, -1);
        part_verdict.assign(rs->part_pad, 0u);
        for (int64_t k = 0; k < rs->part_pad; ++k) never_match_arith(&part_rec[k], &part_wtop[k]);
        for (int c = 0; c < rs->n_classes; ++c)
            for (size_t j = 0; j < lists[c].size(); ++j) {
                const int64_t k = lists[c][j], at = rs->class_off[c] + (int64_t)j;
                part_rec[at] = hq[k];
                part_wtop[at] = hw[k];
                part_orig[at] = (int32_t)k;
                part_verdict[at] = (uint32_t)k | ((uint32_t)(ha[k] & 1u) << 31);
            }
        part_class_of = class_of;
        part_lists = std::move(lists);
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dev_malloc(&rs->d_clamp, rs->n_pad * sizeof(RecClamp));
    if (e == cudaSuccess) e = dev_malloc(&rs->d_cmp, rs->n_pad * sizeof(RecCmp));
    if (e == cudaSuccess) e = dev_malloc(&rs->d_arith, rs->n_pad * sizeof(RecArith));
    if (e == cudaSuccess) e = dev_malloc(&rs->d_wtop, rs->n_pad * sizeof(uint32_t));
    if (e == cudaSuccess) e = dev_malloc(&rs->d_range, rs->n_pad * sizeof(RecRange));
    if (e == cudaSuccess) e = dev_malloc(&rs->d_range_wtop, rs->n_pad * sizeof(uint32_t));
    if (e == cudaSuccess) e = dev_malloc(&rs->d_part, rs->part_pad * sizeof(RecArith));
    if (e == cudaSuccess) e = dev_malloc(&rs->d_part_wtop, rs->part_pad * sizeof(uint32_t));
    if (e == cudaSuccess) e = dev_malloc(&rs->d_part_orig, rs->part_pad * sizeof(int32_t));
    if (e == cudaSuccess) e = dev_malloc(&rs->d_part_verdict, rs->part_pad * sizeof(uint32_t));
    if (e == cudaSuccess) e = dev_malloc(&rs->d_class_of, 256);
    if (e == cudaSuccess) e = dev_malloc(&rs->d_action, rs->n_pad);
    if (e == cudaSuccess) e = dev_malloc(&rs->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemcpy(rs->d_clamp, hc.data(), rs->n_pad * sizeof(RecClamp), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(rs->d_cmp, hm.data(), rs->n_pad * sizeof(RecCmp), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(rs->d_arith, hq.data(), rs->n_pad * sizeof(RecArith), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(rs->d_wtop, hw.data(), rs->n_pad * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(rs->d_range, hr.data(), rs->n_pad * sizeof(RecRange), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(rs->d_range_wtop, hrw.data(), rs->n_pad * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(rs->d_part, part_rec.data(), rs->part_pad * sizeof(RecArith), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(rs->d_part_wtop, part_wtop.data(), rs->part_pad * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(rs->d_part_orig, part_orig.data(), rs->part_pad * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(rs->d_part_verdict, part_verdict.data(), rs->part_pad * sizeof(uint32_t),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(rs->d_class_of, part_class_of.data(), 256, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(rs->d_action, ha.data(), rs->n_pad, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(rs->d_status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = build_filter(rules, part_lists, part_class_of, rs);
    if (e != cudaSuccess) {
        fw_ruleset_destroy(rs);
        cudaGetLastError();
        return set_status(cuda_status(e));
    }
    *out = rs;
    return FW_OK;
}

extern "C" int fw_ruleset_partition(const fw_ruleset *rs, int32_t *n_classes, int32_t *key_field,
                                    int32_t *key_bits) {
    if (rs == nullptr || n_classes == nullptr || key_field == nullptr || key_bits == nullptr)
        return set_status(FW_EINVAL);
    *n_classes = rs->n_classes;
    *key_field = rs->key_field;
    *key_bits = rs->key_bits;
    return FW_OK;
}

extern "C" int fw_ruleset_filter(const fw_ruleset *rs, int32_t *words, int64_t *bytes) {
    if (rs == nullptr || words == nullptr || bytes == nullptr) return set_status(FW_EINVAL);
    *words = rs->filter_words;
    *bytes = rs->filter_bytes;
    return FW_OK;
}

extern "C" int fw_selftest_fail_alloc(int64_t n) {
    g_fail_after.store(n < 0 ? -1 : n, std::memory_order_relaxed);
    return FW_OK;
}

extern "C" int fw_partition_plan(const fw_rule *rules, int64_t n, int32_t granule, int32_t *n_classes,
                                 int32_t *key_field, int32_t *key_bits, int64_t *class_len, uint8_t *proto_class) {
    static_assert(FW_MAX_CLASSES == kMaxClasses, "public class bound");
    if (n < 0 || (n > 0 && rules == nullptr) || n > (int64_t(1) << 30) || granule < 1 || n_classes == nullptr ||
        key_field == nullptr || key_bits == nullptr)
        return set_status(FW_EINVAL);
    for (int64_t k = 0; k < n; ++k) {
        const int s = validate_rule(rules[k]);
        if (s != FW_OK) return set_status(s);
    }
    std::vector<uint8_t> class_of;
    std::vector<std::vector<int64_t>> lists;
    int kf = 0, kb = 0;
    partition_lists(rules, n, granule, class_of, lists, kf, kb);
    *n_classes = (int32_t)lists.size();
    *key_field = kf;
    *key_bits = kb;
    if (class_len != nullptr)
        for (int c = 0; c < kMaxClasses; ++c) class_len[c] = c < (int)lists.size() ? (int64_t)lists[c].size() : 0;
    if (proto_class != nullptr)
        for (int p = 0; p < 256; ++p) proto_class[p] = class_of[p];
    return FW_OK;
}

extern "C" fw_ruleset *fw_ruleset_create(const fw_rule *rules, int64_t n) {
    fw_ruleset *rs = nullptr;
    fw_ruleset_create_ex(rules, n, &rs);
    return rs;
}

extern "C" void fw_ruleset_destroy(fw_ruleset *rs) {
    if (rs == nullptr) return;
    if (rs->d_clamp) cudaFree(rs->d_clamp);
    if (rs->d_cmp) cudaFree(rs->d_cmp);
    if (rs->d_arith) cudaFree(rs->d_arith);
    if (rs->d_wtop) cudaFree(rs->d_wtop);
    if (rs->d_range) cudaFree(rs->d_range);
    if (rs->d_range_wtop) cudaFree(rs->d_range_wtop);
    if (rs->d_part) cudaFree(rs->d_part);
    if (rs->d_part_wtop) cudaFree(rs->d_part_wtop);
    if (rs->d_part_orig) cudaFree(rs->d_part_orig);
    if (rs->d_part_verdict) cudaFree(rs->d_part_verdict);
    if (rs->d_class_of) cudaFree(rs->d_class_of);
    if (rs->d_action) cudaFree(rs->d_action);
    if (rs->d_status) cudaFree(rs->d_status);
    if (rs->d_filter) cudaFree(rs->d_filter);
    delete rs;
}

extern "C" int64_t fw_ruleset_size(const fw_ruleset *rs) { return rs ? rs->n : -1; }
extern "C" int64_t fw_ruleset_first_catch_all(const fw_ruleset *rs) { return rs ? rs->first_catch_all : -1; }

extern "C" int fw_ruleset_check(fw_ruleset *rs) {
    if (rs == nullptr) return set_status(FW_EINVAL);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return set_status(cuda_status(e));
    unsigned st = 0;
    e = cudaMemcpy(&st, rs->d_status, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_status(cuda_status(e));
    if (st != 0) {
        cudaMemset(rs->d_status, 0, sizeof(unsigned));
        return set_status((st & kStatusTimeout) ? FW_ETIMEOUT : FW_ECUDA);
    }
    return FW_OK;
}

extern "C" int fw_last_status(void) { return g_last_status; }

extern "C" const char *fw_status_string(int s) {
    switch (s) {
        case FW_OK: return "ok";
        case FW_EINVAL: return "invalid argument";
        case FW_ENOMEM: return "out of memory";
        case FW_ECUDA: return "CUDA error";
        case FW_EALIGN: return "misaligned buffer";
        case FW_ETIMEOUT: return "bounded device wait timed out";
        case FW_EBUSY: return "busy: no capacity for more work";
        case FW_ERANGE: return "size exceeds the call's fixed limit";
        default: return "unknown status";
    }
}

extern "C" int fw_abi_version(void) { return 1; }
extern "C" int fw_rule_size(void) { return (int)sizeof(fw_rule); }
