// First-match scan kernels and the fw_classify / fw_classify_ex entry points.
//
// Packet split (Sec. IV.A, data-parallel): every worker holds the whole rule
// list and each packet is compared with it by one thread, in list order,
// stopping at the first match. Here a persistent block keeps a prefix of the
// canonical rule records resident in shared memory, brought in by 1-D TMA bulk
// copies in 256-rule chunks, each with its own mbarrier; a warp waits for a
// chunk only when one of its packets first reaches it. All lanes of a warp
// read the same rule at the same time (a broadcast shared-memory load), so one
// load feeds 32 packet checks. Rules past the resident prefix are read from
// global memory (L1/L2 cached) the same way.
//
// Rule split (Sec. IV.B function-parallel, Sec. IV.C hybrid): the rule list is
// divided among workers and the per-packet combine is the minimum matching
// index (first match, Sec. I). Lane l of a warp tests rule 32c + l of chunk c;
// __ballot_sync + __ffs gives the chunk's first match, i.e. the warp-level
// minimum. A block-level minimum (shared-memory atomicMin) combines the warps
// of a block that split one packet group's chunks; a grid-level minimum
// (global atomicMin into stream-ordered scratch, then a finalize pass)
// combines blocks that own different rule slices.
#include <algorithm>
#include <climits>
#include <cstring>

#include "fw_scan.cuh"

namespace fwk {

// ------------------------------------------------------------ packet split kernels
// Lockstep form: persistent grid; each thread takes packet quads (4
// consecutive packets) in a grid-stride loop and scans them one after another.
template <class Pol, bool VEC, bool PART>
__global__ void __launch_bounds__(1024) k_packet_split(ScanParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    // a failed prefix wait leaves every rule to be read from global memory
    const bool staged = stage_rules<Pol>(smem, p);
    const int n_smem = staged ? p.n_smem : 0;
    const typename Pol::View sv = Pol::smem_view(smem, p.n_smem);
    const typename Pol::View gv = Pol::global_view(p);
    const int64_t nq = (p.n + 3) / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += stride) {
        typename Pol::Pk pk[4];
        int cnt;
        load_quad<Pol, VEC>(p.h, p.n, q, pk, cnt);
        int idx[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if constexpr (PART) {
                // the packet's partition class picks its sub-list
                const int c = (int)part_class(__ldg(p.class_of + (pkt_proto<Pol>(pk[j]) & 0xFFu)), p.key_field,
                                              p.key_bits, pk[j].src, pk[j].dst);
                const int off = p.class_off[c];
                const int r = scan_range<Pol>(pk[j], 0, p.class_len[c], shifted_view<Pol>(sv, off),
                                              max(0, n_smem - off), shifted_view<Pol>(gv, off), p.one);
                idx[j] = r < 0 ? -1 : __ldg(p.orig + off + r);
            } else {
                const int r = scan_range<Pol>(pk[j], 0, p.n_scan, sv, n_smem, gv, p.one);
                idx[j] = r < 0 ? -1 : r;
            }
        }
        store_quad<VEC>(p, q, idx, cnt);
    }
    if (!staged) drain_rules<Pol>(smem, p);
}

// Compacting form. Each warp takes a batch of `batch` packets into its own
// shared-memory queue and scans the queue segment by segment over the rule
// list (first segment seg0 rules, then doubling). After each group of 32
// queue entries, packets decided in the segment write their verdicts and the
// undecided ones are packed to the front of the queue (ballot + popc), so the
// next segment runs on dense groups of still-undecided packets instead of
// lanes idling behind the slowest packet of a warp.
template <class Pol, bool VEC, bool PART, int PPL>
__device__ __forceinline__ void compact_body(const ScanParams &p) {
    extern __shared__ __align__(128) unsigned char smem[];
    const bool staged = stage_rules<Pol>(smem, p);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int B = p.batch;
    const size_t qoff = ((size_t)p.n_smem * Pol::bytes_per_rule() + (size_t)(p.n_smem / kChunkRules) * 8 + 15) / 16 * 16;
    uint4 *Q = reinterpret_cast<uint4 *>(smem + qoff) + (size_t)warp * B;
    int *wc = reinterpret_cast<int *>(smem + qoff + (size_t)nw * B * sizeof(uint4)) + warp * 2 * kMaxClasses;
    // block-shared tables (PART only): protocol -> class, and the sub-list offsets / lengths
    uint8_t *tabs = smem + qoff + (size_t)nw * (B * sizeof(uint4) + 2 * kMaxClasses * sizeof(int));
    int32_t *cls_off = reinterpret_cast<int32_t *>(tabs);
    int32_t *cls_len = cls_off + kMaxClasses;
    uint8_t *class_tab = tabs + 2 * kMaxClasses * sizeof(int32_t);
    if constexpr (PART) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) class_tab[i] = p.class_of[i];
        if (threadIdx.x < kMaxClasses) {
            cls_off[threadIdx.x] = p.class_off[threadIdx.x];
            cls_len[threadIdx.x] = p.class_len[threadIdx.x];
        }
        __syncthreads();
    }
    BatchTarget<Pol> t;
    t.h = p.h;
    t.n = p.n;
    t.sv = Pol::smem_view(smem, p.n_smem);
    t.gv = Pol::global_view(p);
    t.n_smem = staged ? p.n_smem : 0;  // a failed prefix wait leaves every rule to global memory
    t.n_scan = p.n_scan;
    t.n_classes = p.n_classes;
    t.key_field = p.key_field;
    t.key_bits = p.key_bits;
    t.class_off = cls_off;
    t.class_len = cls_len;
    t.class_of = class_tab;
    t.orig = p.orig;
    t.verdict = p.verdict;
    t.action = p.action;
    t.out_idx = p.out_idx;
    t.out_act = p.out_act;
    t.seg0 = p.seg0;
    t.one = p.one;
    // packets per batch: the two-packet form keeps queue room for one pad per class
    const int P = PPL == 2 ? B - ((p.n_classes + 3) & ~3) : B;
    const int64_t nb = (p.n + P - 1) / P;
    for (int64_t b = (int64_t)blockIdx.x * nw + warp; b < nb; b += (int64_t)gridDim.x * nw) {
        const int cnt = (int)min((int64_t)P, p.n - b * P);
        if constexpr (PPL == 2) {
            static_assert(PART, "two packets per lane needs the protocol partition");
            run_batch_pairs<Pol, VEC>(t, b * P, cnt, Q, wc, lane);
        } else {
            run_batch<Pol, VEC, PART>(t, b * P, cnt, Q, wc, lane);
        }
    }
    if (!staged) drain_rules<Pol>(smem, p);
}

template <class Pol, bool VEC, bool PART>
__global__ void __launch_bounds__(1024) k_packet_split_compact(ScanParams p) {
    compact_body<Pol, VEC, PART, 1>(p);
}

// Dense form: two 768-thread blocks per SM (48 resident warps, at most 42
// registers a thread) instead of one 1,024-thread block (32 warps).
template <class Pol, bool VEC, bool PART>
__global__ void __launch_bounds__(768, 2) k_packet_split_compact_dense(ScanParams p) {
    compact_body<Pol, VEC, PART, 1>(p);
}

// Two packets per lane in every scan group (each rule load feeds both; two
// independent test chains per lane), one 1,024-thread block per SM.
template <class Pol, bool VEC, bool PART>
__global__ void __launch_bounds__(1024) k_packet_split_compact_x2(ScanParams p) {
    compact_body<Pol, VEC, PART, 2>(p);
}

constexpr int64_t kCompactMinPackets = int64_t(1) << 20;  // default packet split compacts from this batch size
constexpr int64_t kCompactMidPackets = int64_t(3) << 15;  // ... and the partitioned scan, in small blocks, from this
constexpr int64_t kMidMaxPackets = int64_t(1) << 22;      // largest batch given the small-block shape by default

// ------------------------------------------------------------ host side
int sm_count(int dev) {
    static int cached[64] = {0};
    if (dev < 0 || dev >= 64) return 148;
    if (cached[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 148;
    }
    return cached[dev];
}

static bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

template <class K>
static cudaError_t ensure_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int launch_packet_split(const fw_ruleset *rs, const HdrPtrs &h, int64_t n, int32_t *out_idx, uint8_t *out_act,
                        cudaStream_t st, const fw_config &cfg) {
    if (cfg.filter < 0 || cfg.filter > 2) return FW_EINVAL;
    // The bucket filter (fw_filter.cu): on request, or by default when the rule set has one and
    // nothing but the launch shape is configured.
    const bool shape_only = cfg.smem_rules == 0 && cfg.packets_per_group == 0 && cfg.rule_slices == 0 &&
                            cfg.compact == 0 && (cfg.predicate == 0 || cfg.predicate == FW_PRED_ARITH) &&
                            cfg.segment_rules == 0 && cfg.partition == 0 && cfg.lane_packets == 0;
    if (cfg.filter == 1 || (cfg.filter == 0 && shape_only && rs->filter_words > 0))
        return launch_filter(rs, h, n, out_idx, out_act, st, cfg.block_threads, cfg.blocks_per_sm, cfg.lane_packets);
    ScanParams p;
    std::memset(&p, 0, sizeof(p));
    const int pred = cfg.predicate == 0 ? FW_PRED_ARITH : cfg.predicate;
    if (cfg.partition < 0 || cfg.partition > 2) return FW_EINVAL;
    if (cfg.partition == 1 && pred != FW_PRED_ARITH) return FW_EINVAL;
    if (cfg.compact < 0 || cfg.compact > 2) return FW_EINVAL;
    // Default: compaction for large batches; small batches need every thread
    // they can get, so they take the lockstep form with smaller blocks.
    // Default decomposition by batch size (times on the 10K-rule list): the lockstep scan for
    // small batches; the compacting scan of the protocol partition from 98,304 packets, up to
    // 2^22 in 128-thread blocks, eight per SM, where it beats both lockstep and the 1,024-thread
    // form (2^19: 15.0 vs 29.1 and 18.9 us; 2^22: 78.9 vs 148.0 and 82.0 us), and in
    // 1,024-thread blocks above (2^24: 269 vs 298 us); every compacting form from 2^20.
    const bool mid_ok = pred == FW_PRED_ARITH && cfg.partition != 2 && n >= kCompactMidPackets;
    const bool compact = cfg.compact == 1 || (cfg.compact == 0 && (n >= kCompactMinPackets || mid_ok));
    // Protocol partition (stored for the arithmetic form only): default on in
    // the compacting kernel, which sorts each warp's batch by class so that a
    // warp's lanes share one sub-list; in the lockstep kernel lanes of a warp
    // would walk different sub-lists, so there it is used only on request.
    const bool part = pred == FW_PRED_ARITH && (cfg.partition == 1 || (cfg.partition == 0 && compact));
    int rec_bytes;
    if (pred == FW_PRED_CLAMP) {
        p.rec = rs->d_clamp;
        rec_bytes = (int)sizeof(RecClamp);
    } else if (pred == FW_PRED_CMP) {
        p.rec = rs->d_cmp;
        rec_bytes = (int)sizeof(RecCmp);
    } else if (pred == FW_PRED_ARITH) {
        p.rec = part ? (const void *)rs->d_part : (const void *)rs->d_arith;
        rec_bytes = (int)PolArith::bytes_per_rule();
    } else if (pred == FW_PRED_RANGE) {
        p.rec = rs->d_range;
        rec_bytes = (int)PolRange::bytes_per_rule();
    } else {
        return FW_EINVAL;
    }
    p.wtop = pred == FW_PRED_RANGE ? rs->d_range_wtop : (part ? rs->d_part_wtop : rs->d_wtop);
    p.action = rs->d_action;
    const int64_t stored = part ? rs->class_off[kMaxClasses - 1] + rs->class_len[kMaxClasses - 1]
                                : (rs->n_eff + 3) / 4 * 4;
    p.n_scan = (int)stored;
    if (part) {
        p.n_classes = rs->n_classes;
        p.key_field = rs->key_field;
        p.key_bits = rs->key_bits;
        for (int c = 0; c < kMaxClasses; ++c) {
            p.class_off[c] = rs->class_off[c];
            p.class_len[c] = rs->class_len[c];
        }
        p.class_of = rs->d_class_of;
        p.orig = rs->d_part_orig;
        p.verdict = rs->d_part_verdict;
    }
    const int need_all = (int)((p.n_scan + kChunkRules - 1) / kChunkRules * kChunkRules);
    const bool auto_mid = compact && part && n <= kMidMaxPackets && cfg.block_threads <= 0 &&
                          cfg.blocks_per_sm <= 0 && cfg.lane_packets != 1;
    int threads = cfg.block_threads > 0 ? cfg.block_threads : (compact ? (auto_mid ? 128 : 1024) : 512);
    if (cfg.block_threads <= 0 && !compact) {
        // at least two blocks per SM when the batch allows it
        const int64_t nq = (n + 3) / 4;
        const int64_t t = nq / (2 * (int64_t)sm_count(rs->device)) / 32 * 32;
        threads = (int)std::max<int64_t>(64, std::min<int64_t>(512, t));
    }
    const int per_sm = cfg.blocks_per_sm > 0 ? cfg.blocks_per_sm : (compact ? (auto_mid ? 8 : 1) : 2);
    if (threads % 32 != 0 || threads > 1024) return FW_EINVAL;
    if (cfg.lane_packets < 0 || cfg.lane_packets > 2) return FW_EINVAL;
    // Compacting forms: one 1,024-thread block per SM by default; "dense" = the one-packet
    // kernel for two or more blocks of at most 768 threads per SM. With the protocol partition
    // the default gives each lane two packets per group (every rule load feeds two checks),
    // unless a dense shape was asked for.
    const bool dense = compact && cfg.lane_packets != 2 && !auto_mid && threads <= 768 && per_sm >= 2;
    const bool lane2 = compact && part && (cfg.lane_packets == 2 || (cfg.lane_packets == 0 && !dense));
    // the two-packet kernel is built for 64 registers a thread: at most 1,024 threads per SM
    if (lane2 && (int64_t)threads * per_sm > 1024) return FW_EINVAL;
    int want = cfg.smem_rules > 0 ? cfg.smem_rules
                                  : (cfg.smem_rules < 0 ? 0 : (compact ? (auto_mid ? 256 : 2048) : 3072));
    want = (want / kChunkRules) * kChunkRules;
    p.n_smem = std::min(want, need_all);
    p.batch = cfg.packets_per_group > 0 ? cfg.packets_per_group : 256;
    if (compact && cfg.packets_per_group <= 0) {
        // a batch too small to fill every resident warp's 256-entry queue takes 128-entry
        // queues: twice the warps get packets (1K rules x 100K packets: 101 blocks on 152 SMs
        // with 256 entries, 201 with 128)
        const int pads = lane2 ? ((rs->n_classes + 3) & ~3) : 0;
        const int64_t warps = (int64_t)sm_count(rs->device) * per_sm * (threads / 32);
        if ((n + warps - 1) / warps <= 128 - pads) p.batch = 128;
    }
    if (compact && (p.batch % 128 != 0 || p.batch > 65536)) return FW_EINVAL;
    // First segment. With two packets per lane a segment boundary (a re-sort of every queued
    // packet) pays only when sub-lists are long enough for a long tail of deep packets: with the
    // longest sub-list up to 2,048 rules one 512-rule segment wins (100K-rule workload, catch-all
    // at 820: 7.24 vs 7.62 ms at 128), beyond that early compaction does (10K rules without a
    // catch-all: 13.8 vs 15.9 ms at 32).
    int longest = 0;
    if (part)
        for (int c = 0; c < rs->n_classes; ++c) longest = std::max(longest, rs->class_len[c]);
    p.seg0 = cfg.segment_rules > 0 ? cfg.segment_rules
                                   : (part ? (lane2 ? (longest > 2048 ? 32 : 512) : 64) : 16);
    if (p.seg0 % 4 != 0) return FW_EINVAL;
    p.one = 1u;
    p.h = h;
    p.n = n;
    p.out_idx = out_idx;
    p.out_act = out_act;
    p.status = rs->d_status;
    size_t smem = (size_t)p.n_smem * rec_bytes + (size_t)(p.n_smem / kChunkRules) * 8;
    if (compact)
        smem = (smem + 15) / 16 * 16 + (size_t)(threads / 32) * (p.batch * sizeof(uint4) + 2 * kMaxClasses * sizeof(int)) +
               2 * kMaxClasses * sizeof(int32_t) + 256;
    if (smem > 227 * 1024) return FW_EINVAL;
    const bool vec = aligned(h.src, 16) && aligned(h.dst, 16) && aligned(h.sport, 8) && aligned(h.dport, 8) &&
                     aligned(h.proto, 4) && aligned(out_idx, 16) && aligned(out_act, 4);
    int64_t blocks = (int64_t)sm_count(rs->device) * per_sm;
    if (compact) {
        const int per_batch = lane2 ? p.batch - ((p.n_classes + 3) & ~3) : p.batch;
        const int64_t nb = (n + per_batch - 1) / per_batch;
        blocks = std::min<int64_t>(blocks, (nb + threads / 32 - 1) / (threads / 32));
    } else {
        const int64_t nq = (n + 3) / 4;
        blocks = std::min<int64_t>(blocks, (nq + threads - 1) / threads);
    }
    blocks = std::max<int64_t>(1, blocks);
    cudaError_t e = cudaSuccess;
#define FW_LAUNCH_PS(KER, POL, V, PT)                                                        \
    do {                                                                                     \
        e = ensure_smem(KER<POL, V, PT>, smem);                                              \
        if (e == cudaSuccess) KER<POL, V, PT><<<(unsigned)blocks, threads, smem, st>>>(p);     \
    } while (0)
#define FW_LAUNCH_PSD(POL, V, PT)                                                            \
    do {                                                                                     \
        if (dense) FW_LAUNCH_PS(k_packet_split_compact_dense, POL, V, PT);                   \
        else FW_LAUNCH_PS(k_packet_split_compact, POL, V, PT);                               \
    } while (0)
#define FW_LAUNCH_PSX(POL, V, PT)                                                            \
    do {                                                                                     \
        if (lane2) FW_LAUNCH_PS(k_packet_split_compact_x2, POL, V, PT);                      \
        else FW_LAUNCH_PSD(POL, V, PT);                                                      \
    } while (0)
#define FW_PICK(KER)                                                                         \
    do {                                                                                     \
        if (pred == FW_PRED_CLAMP) {                                                         \
            if (vec) FW_LAUNCH_PS(KER, PolClamp, true, false); else FW_LAUNCH_PS(KER, PolClamp, false, false); \
        } else if (pred == FW_PRED_CMP) {                                                    \
            if (vec) FW_LAUNCH_PS(KER, PolCmp, true, false); else FW_LAUNCH_PS(KER, PolCmp, false, false); \
        } else if (pred == FW_PRED_RANGE) {                                                  \
            if (vec) FW_LAUNCH_PS(KER, PolRange, true, false); else FW_LAUNCH_PS(KER, PolRange, false, false); \
        } else if (part) {                                                                   \
            if (vec) FW_LAUNCH_PS(KER, PolArith, true, true); else FW_LAUNCH_PS(KER, PolArith, false, true); \
        } else {                                                                             \
            if (vec) FW_LAUNCH_PS(KER, PolArith, true, false); else FW_LAUNCH_PS(KER, PolArith, false, false); \
        }                                                                                    \
    } while (0)
    if (compact) {
        if (pred == FW_PRED_CLAMP) {
            if (vec) FW_LAUNCH_PSD(PolClamp, true, false); else FW_LAUNCH_PSD(PolClamp, false, false);
        } else if (pred == FW_PRED_CMP) {
            if (vec) FW_LAUNCH_PSD(PolCmp, true, false); else FW_LAUNCH_PSD(PolCmp, false, false);
        } else if (pred == FW_PRED_RANGE) {
            if (vec) FW_LAUNCH_PSD(PolRange, true, false); else FW_LAUNCH_PSD(PolRange, false, false);
        } else if (part) {
            if (vec) FW_LAUNCH_PSX(PolArith, true, true); else FW_LAUNCH_PSX(PolArith, false, true);
        } else {
            if (vec) FW_LAUNCH_PSD(PolArith, true, false); else FW_LAUNCH_PSD(PolArith, false, false);
        }
    } else {
        FW_PICK(k_packet_split);
    }
#undef FW_LAUNCH_PSX
#undef FW_LAUNCH_PSD
#undef FW_PICK
#undef FW_LAUNCH_PS
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(cudaGetLastError());
}

}  // namespace fwk

using namespace fwk;

static int classify_impl(const fw_ruleset *rs, const fw_headers *hdrs, int64_t n, int32_t *out_idx,
                         uint8_t *out_act, void *stream, const fw_config *cfg_in) {
    if (rs == nullptr || n < 0 || n > INT_MAX) return FW_EINVAL;
    if (n == 0) return FW_OK;
    if (hdrs == nullptr || hdrs->src == nullptr || hdrs->dst == nullptr || hdrs->sport == nullptr ||
        hdrs->dport == nullptr || hdrs->proto == nullptr || out_idx == nullptr || out_act == nullptr)
        return FW_EINVAL;
    fw_config cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    if (cfg_in != nullptr) cfg = *cfg_in;
    for (int i = 0; i < 4; ++i)
        if (cfg.reserved[i] != 0) return FW_EINVAL;
    if (cfg.mode < FW_MODE_AUTO || cfg.mode > FW_MODE_RULE_SPLIT_GRID) return FW_EINVAL;
    if (cfg.filter < 0 || cfg.filter > 2) return FW_EINVAL;
    const int dev_ok = check_device(rs);
    if (dev_ok != FW_OK) return dev_ok;
    HdrPtrs h{hdrs->src, hdrs->dst, hdrs->sport, hdrs->dport, hdrs->proto};
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    switch (cfg.mode) {
        case FW_MODE_AUTO:
        case FW_MODE_PACKET_SPLIT:
            return launch_packet_split(rs, h, n, out_idx, out_act, st, cfg);
        case FW_MODE_RULE_SPLIT_WARP:
        case FW_MODE_RULE_SPLIT_BLOCK:
        case FW_MODE_RULE_SPLIT_GRID:
            return launch_rule_split(rs, h, n, out_idx, out_act, st, cfg);
        default:
            return FW_EINVAL;
    }
}

extern "C" int fw_classify(const fw_ruleset *rs, const fw_headers *hdrs, int64_t n, int32_t *out_rule_idx,
                           uint8_t *out_action, void *stream) {
    return set_status(classify_impl(rs, hdrs, n, out_rule_idx, out_action, stream, nullptr));
}

extern "C" int fw_classify_ex(const fw_ruleset *rs, const fw_headers *hdrs, int64_t n, int32_t *out_rule_idx,
                              uint8_t *out_action, void *stream, const fw_config *cfg) {
    return set_status(classify_impl(rs, hdrs, n, out_rule_idx, out_action, stream, cfg));
}

// A wait that nothing completes: the bounded wait must give up and report.
__global__ void k_selftest_wait(unsigned *status, uint64_t limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, status, limit_ns);
}

extern "C" int fw_selftest_wait_timeout(fw_ruleset *rs, int64_t limit_ns, void *stream) {
    if (rs == nullptr || limit_ns < 1000 || limit_ns > 1000000000) return set_status(FW_EINVAL);
    k_selftest_wait<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(rs->d_status, (uint64_t)limit_ns);
    return set_status(cuda_status(cudaGetLastError()));
}

