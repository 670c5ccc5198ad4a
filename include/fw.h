/*
 * fw.h -- C ABI of the GB300 first-match packet classifier.
 *
 * The operation (Sec. I and Sec. IV of "Parallel Firewalls on General-Purpose
 * Graphics Processing Units"): every packet is compared with an ordered rule
 * list; the first rule that matches decides its action, and a packet that no
 * rule matches is dropped (iptables first-match with default deny, Sec. I).
 * A rule is a 5-tuple -- source and destination address, source and
 * destination port, protocol -- plus an action, and a field that a rule does
 * not specify matches every value (Sec. IV). Two decompositions are offered
 * (Sec. IV.A data-parallel: packets split across workers, each holding the
 * whole rule list; Sec. IV.B/C function-parallel and hybrid: the rule list
 * split across workers, combined per packet by taking the smallest matching
 * rule index).
 *
 * Conventions for every entry point:
 *  - Integers are host byte order. Addresses are uint32, ports uint16,
 *    protocol uint8.
 *  - Device pointers are plain CUDA device (or managed) addresses on the
 *    current device; host pointers are ordinary host memory (pinned memory
 *    is faster where noted). No entry point takes ownership of a caller
 *    buffer.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Device-pointer calls are asynchronous with respect to the host:
 *    they enqueue work on `stream` and return; buffers must stay valid until
 *    that work completes.
 *  - Every call that can fail returns an int status: FW_OK (0) or a negative
 *    FW_E* code; nothing is thrown across the ABI. Argument errors are
 *    detected on the host before any work is enqueued.
 *  - There is no CPU fallback: all classification runs in CUDA kernels.
 */
#ifndef FW_H_
#define FW_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define FW_OK        0
#define FW_EINVAL   (-1)  /* bad argument: null pointer, negative size, prefix > 32, lo > hi, bad action/mode */
#define FW_ENOMEM   (-2)  /* device or pinned host allocation failed */
#define FW_ECUDA    (-3)  /* a CUDA runtime call or kernel launch failed */
#define FW_EALIGN   (-4)  /* a buffer is not aligned as the call requires */
#define FW_ETIMEOUT (-5)  /* a bounded device-side wait gave up (see fw_ruleset_check) */
#define FW_EBUSY    (-6)  /* the object cannot take more work now (serving admission) */
#define FW_ERANGE   (-7)  /* a size exceeds a fixed limit of the call */

/* ------------------------------------------------------------------ actions */
#define FW_DROP   0
#define FW_ACCEPT 1

/*
 * One rule as the caller supplies it (24 bytes, Sec. IV 5-tuple + action).
 *  src_addr/dst_addr + src_prefix/dst_prefix: the rule matches addresses whose
 *      top `prefix` bits equal those of the rule's address; prefix 0 matches
 *      every address; bits below the prefix are ignored. prefix must be <= 32.
 *  sport_lo..sport_hi, dport_lo..dport_hi: inclusive port ranges; lo <= hi;
 *      [0, 65535] is the wildcard, [p, p] an exact port.
 *  proto, proto_any: proto_any != 0 matches every protocol, otherwise only
 *      `proto` (protocol 0 is an ordinary value).
 *  action: FW_DROP or FW_ACCEPT.
 */
typedef struct fw_rule {
    uint32_t src_addr;
    uint32_t dst_addr;
    uint16_t sport_lo, sport_hi;
    uint16_t dport_lo, dport_hi;
    uint8_t  src_prefix, dst_prefix;
    uint8_t  proto, proto_any;
    uint8_t  action;
    uint8_t  reserved[3];          /* must be zero */
} fw_rule;

/*
 * A batch of n packet headers, structure of arrays, one element per packet.
 * For the fastest path src/dst should be 16-byte aligned, sport/dport 8-byte
 * and proto 4-byte aligned; other alignments are accepted and take a scalar
 * load path.
 */
typedef struct fw_headers {
    const uint32_t *src;
    const uint32_t *dst;
    const uint16_t *sport;
    const uint16_t *dport;
    const uint8_t  *proto;
} fw_headers;

/* Decomposition selector for fw_classify_ex. */
#define FW_MODE_AUTO             0  /* library picks (packet split unless configured otherwise) */
#define FW_MODE_PACKET_SPLIT     1  /* Sec. IV.A: one thread per packet walks the whole list */
#define FW_MODE_RULE_SPLIT_WARP  2  /* Sec. IV.B/C at warp scale: lanes split 32-rule chunks, ballot picks the first */
#define FW_MODE_RULE_SPLIT_BLOCK 3  /* Sec. IV.C hybrid: a block per packet group, its warps split the rules, block min */
#define FW_MODE_RULE_SPLIT_GRID  4  /* Sec. IV.B: rule slices across blocks, global atomic-min combine */

/* Encodings of the field tests (fw_config.predicate); both give identical results. */
#define FW_PRED_CLAMP 1  /* port ranges as a 16x2 clamp, proto under a mask */
#define FW_PRED_CMP   2  /* port ranges as unsigned subtract-and-compare */
#define FW_PRED_ARITH 3  /* port ranges as multiply-add + compare, protocol folded into dport (default) */
#define FW_PRED_RANGE 4  /* every field (prefixes too) as multiply-add + compare */

/*
 * Launch configuration. Zero in any field means "library default".
 *  mode:              one of FW_MODE_*.
 *  block_threads:     threads per block (multiple of 32; <= 1024 for packet
 *                     split, <= 512 for rule split). Defaults: compacting packet
 *                     split 1024 (128 for partitioned batches of 98,304 to 2^22
 *                     packets), lockstep sized to the batch (<= 512), rule
 *                     split 256 (block mode 512).
 *  blocks_per_sm:     resident blocks per SM for persistent launches (defaults:
 *                     compacting packet split 1 (8 with 128-thread blocks),
 *                     lockstep 2, rule split 4). The two-packet scan allows at
 *                     most 1,024 threads per SM (block_threads x blocks_per_sm).
 *  smem_rules:        rules kept resident in shared memory (packet split;
 *                     defaults 2048 compacting, 256 with 128-thread blocks,
 *                     3072 lockstep; -1 = none).
 *  packets_per_group: rule split: packets handled together by one warp group
 *                     (default 64 for warp and grid mode, 256 for block mode);
 *                     packet split with compaction: queue entries per warp
 *                     batch (multiple of 128, default 256, or 128 when the
 *                     batch would not give every resident warp a full
 *                     256-entry queue; with two packets per lane a batch
 *                     holds up to 4 or 8 fewer packets, room for the class
 *                     pads).
 *  rule_slices:       number of rule slices across the grid (RULE_SPLIT_GRID,
 *                     default 8).
 *  compact:           packet split only: 1 = per-warp queues that re-pack
 *                     undecided packets between rule segments, 2 = plain
 *                     lockstep scan; default: 1 for batches of 2^20 packets or
 *                     more, and for partitioned arithmetic scans from 98,304
 *                     packets; else 2.
 *  predicate:         FW_PRED_CLAMP, FW_PRED_CMP, FW_PRED_ARITH or FW_PRED_RANGE
 *                     (0 = default, the arithmetic form).
 *  segment_rules:     packet split with compaction: rules in the first segment
 *                     (multiple of 4; later segments double). Default: with two
 *                     packets per lane 512, or 32 when the longest class
 *                     sub-list exceeds 2,048 rules; with one packet per lane 64
 *                     (partitioned) or 16 (whole list). Rule split, warp mode
 *                     over the partition when every class sub-list holds at
 *                     most 64 rules: lanes per packet (2, 4, 8 or 16; a warp
 *                     step tests 32 / segment_rules packets against that many
 *                     consecutive rules each; default 4).
 *  partition:         packet split, arithmetic form: 1 = scan the partition
 *                     (default with compaction), 2 = scan the whole list
 *                     (default for the lockstep scan). A rule set keeps, per
 *                     class (a protocol class: the exact protocols its rules
 *                     use most, plus "every other protocol"; split again by
 *                     the top bit(s) of the source or destination address, see
 *                     fw_ruleset_partition), the sub-list of rules that can
 *                     match a packet of that class, in list order; a packet
 *                     scans only its class's sub-list, which contains every
 *                     rule that can match it, so the first match is the same.
 *  lane_packets:      compacting packet split with the partition: packets each
 *                     lane scans at once (1 = one, 2 = two sharing every rule
 *                     load; 0 = default: two, or one when an explicit
 *                     block_threads <= 768 and blocks_per_sm >= 2 select the
 *                     dense form).
 *  filter:            packet split through the bucket filter of the partition:
 *                     per class, bitmaps over its sub-list indexed by the top 8
 *                     bits of the source address, of the destination address
 *                     and the top 4 bits of both ports; a packet tests exactly,
 *                     in list order, only the rules whose three bits are all
 *                     set, which include every rule that contains it, so its
 *                     first match is the same. A rule set has the filter when
 *                     every class sub-list holds at most FW_FILTER_MAX_RULES
 *                     rules and the "every other protocol" class holds no
 *                     exact-protocol rule. Rows of one or two words (sub-lists
 *                     of at most 64 rules) are staged in each block's shared
 *                     memory; wider rows are read from global memory (L1), a
 *                     word at a time up to the packet's first match.
 *                     0 = default: the filter kernel whenever the rule
 *                     set has one and no other field of this struct except
 *                     mode (AUTO or PACKET_SPLIT), block_threads and
 *                     blocks_per_sm is set; 1 = the filter kernel
 *                     (FW_EINVAL if the rule set has none); 2 = never.
 *                     block_threads (<= 512, default 512), blocks_per_sm
 *                     (default 3, or 4 with two packets per thread; fewer
 *                     when the staged filter's shared memory does not fit) and
 *                     lane_packets (packets a thread takes per step with one-
 *                     or two-word rows: 2 or 4; 0 = default, 2 for batches
 *                     under 2^20 packets, else 4) shape its launch.
 */
typedef struct fw_config {
    int32_t mode;
    int32_t block_threads;
    int32_t blocks_per_sm;
    int32_t smem_rules;
    int32_t packets_per_group;
    int32_t rule_slices;
    int32_t compact;
    int32_t predicate;
    int32_t segment_rules;
    int32_t partition;
    int32_t lane_packets;
    int32_t filter;
    int32_t reserved[4];           /* must be zero */
} fw_config;

typedef struct fw_ruleset fw_ruleset;

/* ------------------------------------------------------------ rule sets */
/*
 * Validate, canonicalise (mask addresses, encode wildcards) and copy `n`
 * rules (host array, list order = priority) to device memory on the current
 * device. n may be 0 (every packet is then unmatched). The caller keeps
 * ownership of `rules` and may free it on return. On success *out receives
 * a handle owned by the caller until fw_ruleset_destroy.
 * Errors: FW_EINVAL (null out, n < 0, rules == NULL with n > 0, prefix > 32,
 * lo > hi, action not DROP/ACCEPT, reserved bytes non-zero, n > 2^31-2),
 * FW_ENOMEM, FW_ECUDA. Synchronous.
 */
int fw_ruleset_create_ex(const fw_rule *rules, int64_t n, fw_ruleset **out);

/* Short form: returns the handle, or NULL with the status in fw_last_status(). */
fw_ruleset *fw_ruleset_create(const fw_rule *rules, int64_t n);

/*
 * Free a rule set. No work that uses `rs` may still be in flight (synchronise
 * its streams first). NULL is ignored.
 */
void fw_ruleset_destroy(fw_ruleset *rs);

/* Number of rules, and the index of the first rule that matches every packet (-1 if none). */
int64_t fw_ruleset_size(const fw_ruleset *rs);
int64_t fw_ruleset_first_catch_all(const fw_ruleset *rs);
/*
 * The rule set's partition (arithmetic form; see fw_config.partition): the
 * number of classes, and the address key that splits each protocol class:
 * key_field 0 = none, 1 = source, 2 = destination address, key_bits 0..3 top
 * bits. A packet's class is its protocol class << key_bits | the top key_bits
 * bits of the keyed address. The key is chosen at create time as the one with
 * the shortest mean sub-list.
 */
int fw_ruleset_partition(const fw_ruleset *rs, int32_t *n_classes, int32_t *key_field, int32_t *key_bits);

#define FW_MAX_CLASSES 8

/*
 * The partition of rules[0, n) as given, computed on the host (no device
 * work; usable without a GPU). fw_ruleset_create partitions its rules up to
 * and including the first catch-all with granule 1; fw_lindex_create the rules
 * it indexes with granule 128.
 *  Protocol classes: the up to 7 exact protocols most used by the rules (ties
 *  to the lower value), then "other" for every remaining protocol value. Each
 *  is split by the top key_bits bits of the source (key_field 1) or destination
 *  (2) address, key_bits 1..3, at most FW_MAX_CLASSES classes in all; class =
 *  protocol class << key_bits | key. A class's sub-list keeps, in list order,
 *  the rules that can match one of its packets (protocol "any" or the class's
 *  protocol, or for "other" any protocol without a class of its own; an
 *  address prefix that can hold the key), so a packet's first match (Sec. I)
 *  is the same in its sub-list as in the whole list. The partition itself is
 *  not in the paper: it is this library's way to shorten the scan.
 *  granule: the key (or none) with the lowest mean per-class cost is taken,
 *  the sub-list length for granule 1, else ceil(length / granule) and at least
 *  1. Candidates go source before destination, fewer bits first; a later one
 *  must be strictly lower, and none when no key is.
 *  Outputs: n_classes, key_field, key_bits as fw_ruleset_partition;
 *  class_len (FW_MAX_CLASSES entries, may be NULL): each class's sub-list
 *  length, 0 past n_classes; proto_class (256 entries, may be NULL): the
 *  protocol class of each protocol value.
 * FW_EINVAL for rules NULL with n > 0, n < 0 or n > 2^30, granule < 1, an
 * invalid rule (as fw_ruleset_create), or a NULL n_classes/key_field/key_bits.
 */
int fw_partition_plan(const fw_rule *rules, int64_t n, int32_t granule, int32_t *n_classes, int32_t *key_field,
                      int32_t *key_bits, int64_t *class_len, uint8_t *proto_class);

/* Longest class sub-list a bucket filter covers (rows of up to 256 words). */
#define FW_FILTER_MAX_RULES 8192

/*
 * Bucket filter of the rule set's partition (see fw_config.filter): *words
 * receives the 32-bit words per bitmap row (1 to FW_FILTER_MAX_RULES / 32;
 * 0 when the rule set has no filter: a class sub-list longer than
 * FW_FILTER_MAX_RULES rules, or the "every other
 * protocol" class holding exact-protocol rules), *bytes the size of the
 * filter block each block of the filter kernel stages into shared memory.
 * Host only. FW_EINVAL for NULL arguments.
 */
int fw_ruleset_filter(const fw_ruleset *rs, int32_t *words, int64_t *bytes);

/*
 * The bucket filter a rule set built from these rules would hold (host only,
 * no device memory): the rules up to the first catch-all are partitioned as by
 * fw_partition_plan (granule 1) and, when the partition admits a filter (see
 * fw_ruleset_filter), its filter block is built and copied to `block`.
 * The paper has no counterpart: this exposes the host-side construction so
 * that it can be checked without a GPU.
 *  Outputs: *words (0 = no filter, else the 32-bit words per bitmap row),
 *  *bytes (the block size, 0 without a filter), class_off / class_len
 *  (FW_MAX_CLASSES entries each, may be NULL): first stored record and record
 *  count (a multiple of 4, padding included) of every class sub-list.
 *  Block layout, every part starting on a 16-byte boundary, nc classes,
 *  W words per row, R stored records: the bitmap rows, [class][table][256]
 *  rows of W uint32 words (table 0 indexed by the source address's top 8
 *  bits, table 1 by the destination's, table 2 by (sport >> 12) << 4 |
 *  (dport >> 12); row bit j = record j of the class sub-list); one uint4 per
 *  class (first stored record, exact mask low and high word, 0; exact bit j:
 *  the record needs no exact test); R exact-test records of two uint4
 *  ({saddr & smask, smask, daddr & dmask, dmask} and {-sport_lo,
 *  sport_hi - sport_lo, -dport_lo, dport_hi - dport_lo}, mod 2^32); R verdict
 *  words (original rule index | action << 31); the 256-byte protocol ->
 *  protocol class table; for W >= 32, row summaries, [class][table][256]
 *  rows of ceil(W / 32) uint32 words (bit w set when word w of the row is not
 *  zero: a packet reads only the words set in the AND of its three
 *  summaries).
 * FW_EINVAL as fw_partition_plan, or for NULL bytes/words, capacity < 0, or a
 * NULL block with capacity > 0; FW_ERANGE when 0 < capacity < the block size.
 * With capacity 0 only the sizes are returned.
 */
int fw_filter_plan(const fw_rule *rules, int64_t n, void *block, int64_t capacity, int64_t *bytes,
                   int32_t *words, int32_t *class_off, int32_t *class_len);

/*
 * Synchronise the device and report whether any kernel that used `rs` gave
 * up on a bounded wait since the last check (FW_ETIMEOUT; the flag is then
 * cleared) or a CUDA error is pending (FW_ECUDA).
 */
int fw_ruleset_check(fw_ruleset *rs);

/* ------------------------------------------------------------ classify */
/*
 * Classify n packets (device SoA `hdrs`) against `rs`:
 *   out_rule_idx[i] = smallest k whose rule matches packet i, or -1;
 *   out_action[i]   = action of that rule, or FW_DROP when out_rule_idx[i] = -1.
 * out_rule_idx (int32[n]) and out_action (uint8[n]) are caller-owned device
 * buffers. n = 0 is a no-op. Asynchronous on `stream`; no allocation.
 * Errors: FW_EINVAL (null handle/pointer with n > 0, n < 0, n > 2^31-1), FW_ECUDA.
 */
int fw_classify(const fw_ruleset *rs, const fw_headers *hdrs, int64_t n,
                int32_t *out_rule_idx, uint8_t *out_action, void *stream);

/*
 * As fw_classify with an explicit decomposition / launch configuration
 * (cfg may be NULL for defaults). FW_MODE_RULE_SPLIT_GRID takes a stream-
 * ordered scratch allocation of one int32 per packet for the partial minima.
 */
int fw_classify_ex(const fw_ruleset *rs, const fw_headers *hdrs, int64_t n,
                   int32_t *out_rule_idx, uint8_t *out_action, void *stream,
                   const fw_config *cfg);

/* ------------------------------------------------------------ batched plans */
/*
 * Many (rule set, packet batch) jobs in one persistent launch. The paper
 * accumulates a set of packets and checks them in parallel against one rule
 * set (Sec. IV.A) and suggests asynchronous launches to cut per-batch delay
 * (Sec. V); a plan covers any number of rule sets and batches at once. It is
 * built once (device work list of items: runs of up to packets_per_item - 8
 * packets of one job, longest rule sets first) and launched as often as
 * needed; a persistent grid takes items from a counter, so uneven jobs
 * balance. Each job's result is exactly fw_classify's.
 *
 * A job's buffers must stay valid, and keep their addresses, for the life of
 * the plan (the plan stores the pointers; relaunching re-reads the headers and
 * rewrites the outputs).
 */
typedef struct fw_job {
    const fw_ruleset *rs;
    fw_headers hdrs;         /* device SoA headers */
    int64_t n;               /* packets, 0 <= n <= 2^31-1 */
    int32_t *out_rule_idx;   /* device int32[n] */
    uint8_t *out_action;     /* device uint8[n] */
} fw_job;

/*
 * Plan configuration (zero = default). Rule sets fall into n_classes (1..4)
 * size classes by reachable rules: class c takes sets with at most
 * class_max_rules[c] rules (the last class takes the rest). Per class:
 * packets_per_item (queue entries per warp: multiple of 128, <= 4096, default
 * 256; an item carries up to packets_per_item - 8 packets, the rest holds the
 * pads that keep each protocol class region even for the two-packet scan) and
 * segment_rules (first rule segment of the compacting scan, multiple of 4,
 * default 64). block_threads (default 512; blocks_per_sm default 2: the
 * kernel's 64 registers a thread let 1,024 of its threads reside per SM) x
 * max packets_per_item x 16 bytes of shared memory per block must fit in
 * 227 KB.
 */
typedef struct fw_plan_config {
    int32_t block_threads;
    int32_t blocks_per_sm;
    int32_t n_classes;
    int32_t class_max_rules[4];
    int32_t packets_per_item[4];
    int32_t segment_rules[4];
    int32_t reserved[5];
} fw_plan_config;

typedef struct fw_plan fw_plan;

/* Build a plan (synchronous; copies the job list). Errors: FW_EINVAL, FW_ENOMEM, FW_ECUDA. */
int fw_plan_create(const fw_job *jobs, int64_t n_jobs, const fw_plan_config *cfg, fw_plan **out);
/* Enqueue the whole plan on `stream` (a counter reset and one persistent kernel). */
int fw_plan_launch(fw_plan *plan, void *stream);
/*
 * Same work, replayed from a CUDA graph: the first call captures the launch
 * on an internal stream and instantiates the graph (make it outside any
 * capture of the caller's own); every call launches the graph on `stream`.
 */
int fw_plan_launch_graph(fw_plan *plan, void *stream);
/* Number of work items in the plan (-1 for NULL). */
int64_t fw_plan_items(const fw_plan *plan);
/*
 * The kernel a launch of the plan runs (-1 for NULL): 0 the general batched
 * kernel (some job's rule set has no bucket filter: its items use the
 * two-packet scan, queued in shared memory), 2 or 3 the filter-only kernel
 * (every job has a bucket filter; four packets a lane, no shared memory),
 * built for that many resident 512-thread blocks per SM (blocks_per_sm >= 3
 * picks 3, else 2; the launch has blocks_per_sm blocks per SM, default 2).
 */
int fw_plan_kernel(const fw_plan *plan);
/* Free the plan; no launch of it may still be in flight. */
void fw_plan_destroy(fw_plan *plan);

/* ------------------------------------------------------------ serving */
/*
 * Continuous batching of classification requests (a packet batch for one of
 * the server's device-resident rule sets). A scheduler thread owns `slots`
 * streams; whenever one is free it admits the queued requests that fit (at
 * most max_group_requests requests and max_group_packets packets and, in
 * copy mode, free space in a device staging arena of arena_bytes) and
 * launches them together as one persistent batched kernel. A finished group
 * releases its slot and memory at once, so requests that arrive while others
 * run join the next launch and groups overlap on the device. Each request's
 * result is exactly fw_classify's for its batch.
 *
 * Modes: FW_HOST_COPY (default): request buffers are ordinary host memory
 * (pinned for speed); headers are copied in and verdicts out through the
 * arena. FW_HOST_ZEROCOPY: request buffers must be device memory or pinned
 * host memory; the kernel reads and writes them in place (over the host link
 * for host memory) and no arena is used.
 * A request's buffers must stay valid until it is waited for. The server
 * stands in for the paper's queue-to-user-space and reinject loop (Sec. IV,
 * Fig. 1) and realises its asynchronous launches (Sec. V).
 */
typedef struct fw_server_config {
    int32_t mode;                /* FW_HOST_COPY (0 = default) or FW_HOST_ZEROCOPY */
    int32_t slots;               /* groups in flight at once, 1..16 (default 4) */
    int32_t max_group_requests;  /* requests per launch (default 256) */
    int32_t max_pending;         /* queue capacity; submit returns FW_EBUSY beyond it (default 65536) */
    int64_t max_group_packets;   /* packets per launch (default 2^20); also the largest request */
    int64_t arena_bytes;         /* copy mode device staging budget (default 256 MiB) */
    int32_t packets_per_item;    /* queue entries per warp (multiple of 128, default 256); an item carries 8 fewer packets */
    int32_t segment_rules;       /* first rule segment of the compacting scan (default 64) */
    int32_t block_threads;       /* kernel block size (default 512) */
    int32_t items_per_warp;      /* a group launched while others are in flight has at most enough
                                    blocks to give each warp this many work items on average
                                    (default 1: every SM it can use, the lowest latency; larger
                                    leaves SMs to the groups beside it); a group alone on the
                                    device always gets one item a warp */
    int32_t busy_groups;         /* with this many groups in flight (default 2), queued requests
                                    wait to form a full group (max_group_packets queued) or for a
                                    group to complete: under load groups grow, fewer launches */
    int32_t reserved[3];
} fw_server_config;

typedef struct fw_server_stats {
    int64_t submitted, completed, failed, packets;
    int64_t groups;               /* launches */
    int64_t max_group_requests;   /* largest group admitted */
    int64_t max_inflight_groups;  /* most groups on the device at once */
    int64_t arena_high_water;     /* most arena bytes in use at once */
    int64_t pending;              /* queued now */
    int64_t submit_ns;            /* host time spent checking and queueing requests (submit, replay) */
    int64_t launch_ns;            /* scheduler time spent admitting groups and enqueueing their work */
    int64_t complete_ns;          /* scheduler time spent polling groups and completing their requests */
} fw_server_stats;

/* One request of a replayed arrival schedule (fw_server_replay). */
typedef struct fw_request {
    int32_t set;             /* rule set index */
    int32_t status;          /* out: FW_OK or an error */
    fw_headers hdrs;         /* request buffers, as for fw_server_submit */
    int64_t n;
    int32_t *out_rule_idx;
    uint8_t *out_action;
    double arrival_us;       /* in: arrival time after the replay starts */
    double latency_us;       /* out: completion time minus scheduled arrival */
    double submit_lag_us;    /* out: queue entry time minus scheduled arrival (the submitter's own delay) */
} fw_request;

typedef struct fw_server fw_server;

/* Start a server over n_sets rule sets (the caller keeps them alive until destroy). */
int fw_server_create(const fw_ruleset *const *sets, int n_sets, const fw_server_config *cfg, fw_server **out);
/* Finish all queued and running requests, stop the scheduler, free everything. */
void fw_server_destroy(fw_server *sv);
/*
 * Queue a request of n (1..max_group_packets) packets for rule set `set`;
 * *ticket identifies it. Returns at once. FW_EBUSY when the queue is full
 * (max_pending requests queued) or when the ticket issued R submits earlier
 * has not been released by fw_server_wait yet (R: max_pending + slots x
 * max_group_requests, rounded up to a power of two; requests are kept in a
 * ring of R entries), FW_ERANGE when the request can never fit (too many
 * packets, or more arena bytes than the arena has), FW_EINVAL for bad
 * arguments (in zero-copy mode also for buffers the device cannot reach).
 */
int fw_server_submit(fw_server *sv, int set, const fw_headers *hdrs, int64_t n, int32_t *out_rule_idx,
                     uint8_t *out_action, uint64_t *ticket);
/*
 * Wait for a request (timeout_us < 0: no limit); on return other than
 * FW_ETIMEOUT the ticket is released and *latency_us (may be NULL) holds
 * completion minus submit time in microseconds. Returns the request's status.
 */
int fw_server_wait(fw_server *sv, uint64_t ticket, int64_t timeout_us, double *latency_us);
/* Wait until nothing is queued or running (tickets stay valid for fw_server_wait). */
int fw_server_drain(fw_server *sv, int64_t timeout_us);
/*
 * Zero-copy mode: declare that [p, p + bytes) (device memory or pinned host
 * memory) will hold request buffers, so submits whose arrays lie inside it
 * skip the per-call pointer lookups. The buffer must stay allocated until it
 * is unregistered (by its start address) or the server is destroyed.
 * FW_EINVAL if the range is not device accessible as one piece.
 */
int fw_server_register_buffer(fw_server *sv, const void *p, size_t bytes);
int fw_server_unregister_buffer(fw_server *sv, const void *p);
int fw_server_get_stats(fw_server *sv, fw_server_stats *st);
/*
 * Open-loop replay: submit reqs[i] at arrival_us[i] after the call starts
 * (retrying while the queue is full; requests already due are prepared and
 * queued together), then wait for all of them and fill status, latency_us
 * and submit_lag_us. While it submits, the scheduler thread is kept polling
 * instead of sleeping between requests, as under steady traffic; the clock
 * starts once it is awake. Returns FW_OK when every request succeeded.
 */
int fw_server_replay(fw_server *sv, fw_request *reqs, int64_t n, int64_t timeout_us);

/* ------------------------------------------------------- device request queue */
/*
 * Continuous batching with the scheduling on the device. The host writes each
 * request (a packet batch for one of the queue's rule sets) into a ring of
 * descriptors in pinned host memory and publishes it by storing the next
 * ticket into a tail word after the ring; nothing else happens on the host per
 * request. One persistent kernel runs while requests keep coming: four warps
 * of its first block read new descriptors from the ring (up to 128 a pass),
 * split each request into work items (chunk_packets packets, larger when many
 * requests wait) and write them into a device item ring; every other warp
 * claims item tickets from a
 * global counter, classifies its item through the request's bucket filter
 * (the routine of fw_classify's default packet split, Sec. IV.A) and, when it
 * finishes a request's last item, stores the ticket into the request's
 * completion word in pinned host memory, which fw_dqueue_wait polls. Requests
 * that arrive while others run are taken up as soon as the reading warps see
 * them, and items of different requests and rule sets run side by side, so
 * there are no groups and no launch per request. The paper's prototype
 * collects packets, classifies them in one launch and hands the verdicts
 * back (Sec. IV, Fig. 1) and names asynchronous launches as the next step
 * (Sec. V); here the launch outlives the requests.
 *
 * Every device-side wait is bounded by %globaltimer: the reading warps give up
 * after idle_us without a new request (the kernel then exits, and the next
 * submit launches it again, or, when the submit and the exit cross, the
 * first wait that finds the request pending for 50 us; fw_dqueue_stats counts
 * launches and exits), a kernel stops
 * taking requests after life_ms (the host relaunches it), and a worker that
 * waited over 4 x life_ms for its item sets an error flag and exits. While the
 * kernel runs it holds blocks_per_sm x 512 threads on every SM; work on other
 * streams waits for SMs it frees, at the latest idle_us after the last request.
 *
 * Results are exactly fw_classify's for each request. Every rule set must
 * have a bucket filter (fw_ruleset_filter: words > 0). Request buffers must
 * lie in ranges registered with fw_dqueue_register_buffer (device memory or
 * pinned host memory) and stay valid until the request is waited for.
 *
 * fw_dqueue_config (zero = default):
 *  ring:                requests in flight at once, a power of two 64..65536
 *                       (default 4096); a ticket's ring entry is reused only
 *                       after it was waited for.
 *  chunk_packets:       packets per work item while at most 8 requests wait
 *                       in the ring, a multiple of 64 up to 65536 (default
 *                       64); the device takes 4x with up to 128 waiting and
 *                       16x beyond (fewer, larger items under load).
 *  blocks_per_sm:       1 or 2 (default 2) resident 512-thread blocks.
 *  idle_us:             the kernel's idle limit (default 1000).
 *  max_request_packets: largest request (default 65536); the item ring holds
 *                       ring x ceil(max_request_packets / chunk_packets) items
 *                       of 8 bytes, at most 2^26.
 *  life_ms:             the kernel's time limit (default 2000).
 *  poll_ns:             the longest sleep of a waiting worker between polls
 *                       (from 32 ns, doubling; default 2048).
 */
typedef struct fw_dqueue_config {
    int32_t ring;
    int32_t chunk_packets;
    int32_t blocks_per_sm;
    int32_t idle_us;
    int64_t max_request_packets;
    int32_t life_ms;
    int32_t poll_ns;
    int32_t reserved[4];           /* must be zero */
} fw_dqueue_config;

typedef struct fw_dqueue_stats {
    int64_t submitted, completed, packets;
    int64_t launches;              /* persistent-kernel launches */
    int64_t idle_exits;            /* launches that ended because no request came for idle_us */
    int64_t life_exits;            /* launches that ended at life_ms */
    int64_t fed_requests;          /* requests the device took from the ring */
    int64_t fed_items;             /* work items it released */
    int64_t device_status;         /* error flags: 1 = a worker's wait ran out */
    int64_t submit_ns;             /* host time spent in submit */
    int64_t feed_ns, feeds;        /* device time the reading warp spent taking requests, and how
                                      many times it took some */
    int64_t feed_read_ns;          /* the part of feed_ns spent reading ring entries */
    int64_t work_ns, items_done;   /* device time workers spent on items (summed over warps), and
                                      the items (these two and device_status are read while no
                                      launch runs; they keep their last values otherwise) */
} fw_dqueue_stats;

typedef struct fw_dqueue fw_dqueue;

/*
 * Create a queue over n_sets rule sets (kept alive by the caller until
 * destroy; all on the current device). FW_EINVAL for bad arguments, a bad
 * config or a rule set without a bucket filter; FW_ERANGE when the item ring
 * would exceed 2^26 items; FW_ENOMEM, FW_ECUDA. The kernel starts at the first
 * submit.
 */
int fw_dqueue_create(const fw_ruleset *const *sets, int n_sets, const fw_dqueue_config *cfg, fw_dqueue **out);
/* Stop the kernel (it finishes what it has taken), free everything. No request may be pending. */
void fw_dqueue_destroy(fw_dqueue *q);
/*
 * Declare [p, p + bytes) (device memory or pinned host memory of the queue's
 * device) as holding request buffers. FW_EINVAL if the range is not device
 * accessible as one piece.
 */
int fw_dqueue_register_buffer(fw_dqueue *q, const void *p, size_t bytes);
/*
 * Queue a request of n (1..max_request_packets) packets for rule set `set`;
 * returns at once with *ticket. FW_EBUSY when the ticket's ring entry still
 * holds a request not waited for; FW_ERANGE for n above max_request_packets;
 * FW_EINVAL for bad arguments or buffers outside the registered ranges.
 * One thread at a time may submit.
 */
int fw_dqueue_submit(fw_dqueue *q, int set, const fw_headers *hdrs, int64_t n, int32_t *out_rule_idx,
                     uint8_t *out_action, uint64_t *ticket);
/*
 * Wait for a request (timeout_us < 0: no limit). FW_OK: done, the ticket is
 * released and *latency_us (may be NULL) holds completion minus submit time;
 * FW_ETIMEOUT: not done yet (the ticket stays valid); FW_EINVAL for a ticket
 * that is not pending; FW_ECUDA when the kernel failed.
 */
int fw_dqueue_wait(fw_dqueue *q, uint64_t ticket, int64_t timeout_us, double *latency_us);
int fw_dqueue_get_stats(fw_dqueue *q, fw_dqueue_stats *st);
/*
 * Open-loop replay, as fw_server_replay: reqs[i] is submitted at arrival_us[i]
 * after the call starts (retrying while its ring entry is busy), a second
 * host thread records each completion as it happens, and status, latency_us
 * (completion minus scheduled arrival) and submit_lag_us are filled in.
 * Returns FW_OK when every request succeeded.
 */
int fw_dqueue_replay(fw_dqueue *q, fw_request *reqs, int64_t n, int64_t timeout_us);

/* ------------------------------------------------------------ learned index */
/*
 * Decomposition classifier with a learned locator (same result as
 * fw_classify). Each rule field is an interval of its key space (Sec. IV:
 * prefix = address interval, port range, protocol value or all). Per field
 * the key space is cut at every interval end into elementary intervals. The
 * protocol and address key select a class as in fw_classify's partition (the
 * up to 7 exact protocols most used, plus "other", split by the top bits of
 * one address where that shortens the sub-lists; fw_ruleset_partition
 * describes it); per class, row j of a field's bitmap
 * (src, dst, sport, dport) has bit b set when the b-th rule of the class's
 * sub-list covers interval j. A packet's first match (Sec. I) is the rule
 * behind the lowest set bit of the AND of its four rows in its class (five
 * when the class is "other" and holds exact-protocol rules: then a protocol
 * row is ANDed as well, since the class no longer implies the protocol). The
 * interval holding a key is found by a piecewise-linear FP32 model
 * (the key space cut into `segments` equal parts, one line per part fit on
 * the sorted interval ends: least squares or the chord, whichever has the
 * smaller exact error bound) whose stored per-part maximum error
 * bounds an exact integer binary search; the search window is verified with
 * integer compares, and a failed check falls back to a full search (counted
 * in fw_lindex_stats.fallbacks), so no floating-point value decides a match.
 *
 * fw_lindex_config (zero = default):
 *  segments: model parts per field, a power of two <= 65536 (default 4096;
 *            fields with fewer keys use one part per key).
 *  truncate: 1 (default) index only rules up to the first catch-all (no
 *            packet is decided after it); 2 index every rule.
 * Device memory: per class and field (src, dst, sport, dport), rows x
 * ceil(sub-list/128)*16 bytes, rows <= 2 x indexed rules + 1. Create is
 * synchronous and copies `rules`.
 */
typedef struct fw_lindex_config {
    int32_t segments;
    int32_t truncate;
    int32_t reserved[6];
} fw_lindex_config;

typedef struct fw_lindex_stats {
    int64_t rules;          /* rules supplied */
    int64_t rules_indexed;  /* rules in the bitmaps */
    int64_t words_per_row;  /* 32-bit words per bitmap row (the longest class sub-list's) */
    int64_t segments;       /* model parts per field (upper bound) */
    int64_t intervals[5];   /* elementary intervals: src, dst, sport, dport, proto */
    int32_t max_error[5];   /* stored maximum model error per field, in positions */
    int64_t bitmap_bytes;   /* device bytes of all rows */
    int64_t fallbacks;      /* verified windows that failed (0 when the bounds hold) */
    int64_t classes;        /* partition classes (one set of rows each) */
    int32_t key_field;      /* address key of the partition: 0 none, 1 src, 2 dst */
    int32_t key_bits;       /* top address bits in the key */
} fw_lindex_stats;

typedef struct fw_lindex fw_lindex;

int fw_lindex_create(const fw_rule *rules, int64_t n, const fw_lindex_config *cfg, fw_lindex **out);
void fw_lindex_destroy(fw_lindex *li);
/* As fw_classify (device SoA headers, device outputs, asynchronous on stream). */
int fw_lindex_classify(const fw_lindex *li, const fw_headers *hdrs, int64_t n, int32_t *out_rule_idx,
                       uint8_t *out_action, void *stream);
/* Synchronises the device and fills *st. */
int fw_lindex_get_stats(fw_lindex *li, fw_lindex_stats *st);

/* ------------------------------------------------------------ host buffers */
/*
 * Host-ingress path: classify packets whose headers live in HOST memory and
 * return verdicts to host memory. It stands in for the paper's loop of
 * accumulating a batch, copying it to the device, launching and copying the
 * verdict array back (Sec. IV.A/IV.C; Fig. 1 queue and reinject), without a
 * kernel module.
 *
 * A pipeline owns its streams and per-stream device staging buffers of
 * `chunk_packets` packets (0 = 4,194,304). Strategies:
 *   FW_HOST_COPY:     chunks are copied H2D, classified and copied D2H on
 *                     `n_streams` streams (1..8, 0 = 3) so copies of one chunk
 *                     overlap the scan of another. Pinned host buffers are
 *                     needed for the overlap; pageable ones work but serialise.
 *   FW_HOST_ZEROCOPY: the kernels read the headers from, and write verdicts
 *                     to, pinned host memory directly (mapped pages over the
 *                     host link); every buffer must be pinned (page-locked by
 *                     cudaHostAlloc / cudaHostRegister), else FW_EINVAL.
 * fw_classify_host is synchronous: on return the verdicts are in host memory.
 */
#define FW_HOST_COPY     1
#define FW_HOST_ZEROCOPY 2

typedef struct fw_host_pipeline fw_host_pipeline;

int fw_host_pipeline_create(int64_t chunk_packets, int n_streams, fw_host_pipeline **out);
void fw_host_pipeline_destroy(fw_host_pipeline *pl);

/*
 * Classify n packets given in host SoA arrays `host_hdrs`; verdicts go to the
 * host arrays out_rule_idx (int32[n]) and out_action (uint8[n]). `strategy`
 * is FW_HOST_COPY or FW_HOST_ZEROCOPY; cfg as for fw_classify_ex (may be NULL).
 * Errors: FW_EINVAL (null arguments, n < 0, unpinned buffer with
 * FW_HOST_ZEROCOPY), FW_ECUDA.
 */
int fw_classify_host(fw_host_pipeline *pl, const fw_ruleset *rs, const fw_headers *host_hdrs, int64_t n,
                     int32_t *out_rule_idx, uint8_t *out_action, int strategy, const fw_config *cfg);

/* ------------------------------------------------------------ no allocation */
/*
 * Largest batch fw_classify_rule_split_noalloc accepts (packets). Its scratch
 * is a fixed device array of this many int32 values (4 MiB) that every GPU
 * which loads this library keeps until the process exits.
 */
#define FW_NOALLOC_MAX_PACKETS (1 << 20)

/*
 * The paper has no counterpart to this call; it exists for callers that must
 * not allocate device memory while classifying. Examples: a packet path that
 * cannot afford the implicit device synchronisation and latency of
 * cudaMalloc/cudaFree, a service whose GPU memory footprint is fixed when it
 * starts (every later allocation is refused or would compete with other
 * tenants), or code that runs where the stream-ordered allocator has been
 * disabled.
 *
 * Same result as fw_classify_ex with FW_MODE_RULE_SPLIT_GRID (same cfg
 * fields, same launch shape, same kernels), but the per-packet partial minima
 * live in a file-scope device array of FW_NOALLOC_MAX_PACKETS int32 values
 * instead of a per-call allocation. No cudaMalloc, cudaFree or other
 * allocating routine is called. The caller still passes the device headers
 * and the two device output arrays.
 *  - n > FW_NOALLOC_MAX_PACKETS: FW_ERANGE, nothing is launched.
 *  - Other argument errors as fw_classify_ex (FW_EINVAL: also for non-zero
 *    reserved fields, and when the current device is not the rule set's);
 *    cfg may be NULL; mode must be 0 or FW_MODE_RULE_SPLIT_GRID.
 *  - The first call on a device looks up that device's address of the array
 *    (cudaGetSymbolAddress) with the device current and caches it. With the
 *    CUDA runtime's lazy module loading, that first call may also load the
 *    library's kernels and the array itself onto the device, which takes
 *    device memory once. So make one warm-up call per device at start-up,
 *    before any stream capture; later calls allocate nothing.
 *  - Every call on a device shares the one array, and each call re-fills the
 *    part it uses before use, so stale contents from an earlier call never
 *    leak into a result. Two calls whose work overlaps on the GPU (different
 *    streams, or different host threads, without ordering between them) race
 *    on the array and may return wrong verdicts: order them on one stream or
 *    synchronise between them.
 * Asynchronous on `stream` like fw_classify.
 */
int fw_classify_rule_split_noalloc(const fw_ruleset *rs, const fw_headers *hdrs, int64_t n,
                                   int32_t *out_rule_idx, uint8_t *out_action, void *stream,
                                   const fw_config *cfg);

/* ------------------------------------------------------------ measurement */
/*
 * Integer throughput microbenchmark (the paper has no counterpart: it measures
 * the INT32 peak that rule-check rates are reported against, on the GPU the
 * library runs on). Enqueues one kernel on `stream`: `blocks` x `threads`
 * threads, each running `iters` loop trips of 128 independent-chain 32-bit
 * integer instructions with no memory traffic, then one uint32 store per
 * thread into `sink` (device memory, at least blocks*threads uint32, caller
 * owned). kind 0: lop3 only (the integer ALU pipe); kind 1: mad.lo.u32 only
 * (integer multiply-add, issued on the FMA pipe); kind 2: both alternated 1:1
 * (the issue limit when both pipes are fed). *ops_per_launch receives the
 * instruction count of one launch (blocks*threads*iters*128, per-thread ops,
 * i.e. lanes x instructions); the caller times the launch (CUDA events on
 * `stream`) and divides.
 *  - FW_EINVAL: kind outside 0..2, iters outside 1..2^24, blocks outside
 *    1..2^20, threads not a multiple of 32 in 32..512, NULL sink or
 *    ops_per_launch. FW_ECUDA: launch failure.
 */
int fw_int32_peak_launch(int kind, int32_t iters, int32_t blocks, int32_t threads, uint32_t *sink,
                         void *stream, int64_t *ops_per_launch);

/* ------------------------------------------------------------ self test */
/*
 * Failure-path check of the bounded device waits. Launches one block whose
 * thread waits on an mbarrier that nothing will complete, with a limit of
 * `limit_ns` nanoseconds (1e3..1e9); the wait gives up, records the timeout
 * in the rule set's status word and the kernel returns normally, so the CUDA
 * context stays usable. A following fw_ruleset_check(rs) returns FW_ETIMEOUT.
 * The paper has no counterpart; this exists so that tests can exercise the
 * timeout path of the kernels' waits without faulting or hanging a GPU.
 */
int fw_selftest_wait_timeout(fw_ruleset *rs, int64_t limit_ns, void *stream);

/*
 * Test hook for allocation failure, injected on the host (no GPU fault). The
 * (n+1)-th device or pinned host allocation that a create call makes from now
 * on fails once as if memory ran out, and the hook then disarms; n < 0
 * disarms it. Create calls are fw_ruleset_create(_ex), fw_lindex_create,
 * fw_plan_create, fw_server_create and fw_host_pipeline_create. The failing
 * call frees what it holds and returns FW_ENOMEM with a NULL handle.
 * Classify-time scratch (the grid rule split's) is not counted.
 * Process-wide; the counter is atomic, but which of several concurrent creates
 * meets the failure is not defined. Returns FW_OK.
 */
int fw_selftest_fail_alloc(int64_t n);

/* ------------------------------------------------------------ misc */
int fw_last_status(void);                 /* status of the last failed short-form call on this thread */
const char *fw_status_string(int status); /* static string, never NULL */
int fw_abi_version(void);                 /* increments on incompatible ABI changes */
int fw_rule_size(void);                   /* sizeof(fw_rule) == 24 */

#ifdef __cplusplus
}
#endif
#endif /* FW_H_ */
