/*
 * CPU oracle for first-match, default-deny packet classification.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the bench's CPU
 * baseline use it. It shares no code, header, table or helper with the CUDA
 * library; it reads the caller's rule array in its original (unpacked)
 * form and re-derives every field test from the definitions below.
 *
 * What it computes (plain definition, written out):
 *   idx(p)    = min { k in [0, N) : p in S_k }, or -1 if no rule contains p
 *   action(p) = rule[idx(p)].action, or DROP (0) when idx(p) = -1
 * with S_k the product of the per-field sets of rule k:
 *   - source / destination address: all 32-bit values whose top `prefix`
 *     bits equal those of the rule's address; prefix 0 = every address
 *     (Sec. IV: an unspecified field matches every value of that field);
 *   - source / destination port: the inclusive range [lo, hi];
 *   - protocol: the rule's value, or every value when proto_any != 0.
 * First match and default deny are the iptables policy the paper adopts
 * (Sec. I); packets are examined one after another, each against the rules
 * in list order (Sec. I, sequential filtering; Sec. IV "Results and
 * Analysis", the CPU run the parallel models are compared with).
 *
 * depth(p) = idx(p) + 1, or N when unmatched: the number of rules the
 * sequential loop examines for p. The sum over packets is returned.
 *
 * The packet loop may be spread over threads (OpenMP); each packet's result
 * is computed by the same sequential rule loop whatever the thread count.
 */
#include <stdint.h>
#include <stddef.h>

typedef struct {
    uint32_t src_addr;
    uint32_t dst_addr;
    uint16_t sport_lo, sport_hi;
    uint16_t dport_lo, dport_hi;
    uint8_t  src_prefix, dst_prefix;
    uint8_t  proto, proto_any;
    uint8_t  action;
    uint8_t  reserved[3];
} oracle_rule;                      /* 24 bytes, same byte layout as the library's input rule */

/* Address field (Sec. IV): same top `prefix` bits. 64-bit shift so that a
 * prefix of 0 shifts by 32 and compares 0 == 0 (matches every address). */
static int address_matches(uint32_t addr, uint32_t rule_addr, unsigned prefix)
{
    unsigned drop = 32u - prefix;               /* 0..32 low bits ignored */
    uint64_t a = (uint64_t)addr >> drop;
    uint64_t b = (uint64_t)rule_addr >> drop;
    return a == b;
}

/* Port field: inclusive range. */
static int port_matches(uint16_t port, uint16_t lo, uint16_t hi)
{
    return lo <= port && port <= hi;
}

/* Protocol field: one value, or any. */
static int proto_matches(uint8_t proto, uint8_t rule_proto, uint8_t any)
{
    if (any) return 1;
    return proto == rule_proto;
}

static int rule_matches(const oracle_rule *r, uint32_t src, uint32_t dst,
                        uint16_t sport, uint16_t dport, uint8_t proto)
{
    return address_matches(src, r->src_addr, r->src_prefix)
        && address_matches(dst, r->dst_addr, r->dst_prefix)
        && port_matches(sport, r->sport_lo, r->sport_hi)
        && port_matches(dport, r->dport_lo, r->dport_hi)
        && proto_matches(proto, r->proto, r->proto_any);
}

int oracle_abi_version(void) { return 1; }
int oracle_rule_size(void) { return (int)sizeof(oracle_rule); }

/*
 * Classify n packets (SoA host arrays) against n_rules rules (host array in
 * list order). Writes out_idx[i] and out_action[i]; returns sum of depth(p).
 * threads <= 1 runs the plain single-threaded loop.
 */
int64_t oracle_classify(const oracle_rule *rules, int64_t n_rules,
                        const uint32_t *src, const uint32_t *dst,
                        const uint16_t *sport, const uint16_t *dport,
                        const uint8_t *proto, int64_t n,
                        int32_t *out_idx, uint8_t *out_action, int threads)
{
    int64_t total_depth = 0;
    if (threads < 1) threads = 1;
#pragma omp parallel for num_threads(threads) schedule(static) reduction(+ : total_depth) if (threads > 1)
    for (int64_t i = 0; i < n; ++i) {
        int32_t found = -1;
        for (int64_t k = 0; k < n_rules; ++k) {
            if (rule_matches(&rules[k], src[i], dst[i], sport[i], dport[i], proto[i])) {
                found = (int32_t)k;
                break;
            }
        }
        out_idx[i] = found;
        out_action[i] = (found < 0) ? (uint8_t)0 /* DROP: default deny */ : rules[found].action;
        total_depth += (found < 0) ? n_rules : (int64_t)found + 1;
    }
    return total_depth;
}
