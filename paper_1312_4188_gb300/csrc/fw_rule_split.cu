// Rule split (Sec. IV.B function-parallel, Sec. IV.C hybrid): the rule list is
// divided among workers and each packet's results are combined by taking the
// smallest matching rule index (first match, Sec. I). Lane l of a warp holds
// rule 32c + l of chunk c in registers and tests it against one packet at a
// time; __ballot_sync + __ffs gives the chunk's first match, the warp-level
// minimum. A block-level minimum (shared-memory atomicMin) combines the warps
// of a block that split one packet group's chunks (the hybrid); a grid-level
// minimum (global atomicMin into per-packet scratch, then a finalize pass)
// combines blocks that own different rule slices.
//
// Two rule layouts: the partition (default: a packet is tested only against
// its class's sub-list, which holds every rule that can match it, in list
// order, so the first match is the same) and the whole list (on request).
#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>

#include "fw_scan.cuh"

namespace fwk {

// ------------------------------------------------------------ whole-list kernel (clamp records)
struct SplitParams {
    const RecClamp *clamp;
    const uint8_t *action;
    int n_scan;        // rules scanned (multiple of 4; padded records never match)
    int slice_rules;   // rules per slice along gridDim.y (multiple of 32)
    int group;         // packets per group (multiple of 32)
    int gw;            // block mode: warps sharing one packet group (<= warps per block)
    HdrPtrs h;
    int64_t n;
    int32_t *out_idx;
    uint8_t *out_act;
    int32_t *partial;  // grid mode: per-packet minimum across slices (pre-set to kNoMatch)
};

constexpr int kNoMatch = 0x7F7F7F7F;  // byte-fill sentinel, larger than any rule index

// BLOCK = true: all warps of the block share one packet group and split its
// chunks round-robin. BLOCK = false: each warp owns a packet group alone.
// Barrier over the gw warps of packet group g: the warp itself when gw is 1,
// otherwise named barrier 1 + g (barrier 0 is __syncthreads'; at most 8 groups
// share a block when gw >= 2).
__device__ __forceinline__ void group_sync(int gw, int g) {
    if (gw == 1) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(gw * 32) : "memory");
}

template <bool BLOCK>
__global__ void __launch_bounds__(512) k_rule_split(SplitParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int G = p.group;
    // Block mode (the paper's hybrid): gw warps share a packet group and split its rule
    // chunks; a block holds nwarps / gw such groups, each synchronised by its own named
    // barrier (gw is the chunk count when the list is short, so no warp sits idle).
    const int gw = BLOCK ? p.gw : 1;
    const int groups_per_block = nwarps / gw;
    const int my_group = warp / gw;
    if (my_group >= groups_per_block) return;  // warps left over when gw does not divide nwarps
    const int w_in_group = warp % gw;
    const int gt = w_in_group * 32 + lane;  // thread index within the group
    const int gthreads = gw * 32;
    Pkt *stage = reinterpret_cast<Pkt *>(smem) + (size_t)my_group * G;
    int *best = reinterpret_cast<int *>(smem + (size_t)groups_per_block * G * sizeof(Pkt)) + (size_t)my_group * G;

    const int r0 = blockIdx.y * p.slice_rules;
    const int r1 = min(p.n_scan, r0 + p.slice_rules);
    const int64_t n_groups = (p.n + G - 1) / G;
    for (int64_t g = (int64_t)blockIdx.x * groups_per_block + my_group; g < n_groups;
         g += (int64_t)gridDim.x * groups_per_block) {
        const int64_t base = g * G;
        for (int t = gt; t < G; t += gthreads) {
            const int64_t i = base + t;
            if (i < p.n) {
                stage[t] = {p.h.src[i], p.h.dst[i], ports_of(p.h.sport[i], p.h.dport[i]), p.h.proto[i]};
                best[t] = INT_MAX;
            } else {
                stage[t] = {0, 0, 0, 0};
                best[t] = -1;  // no packet: never pending
            }
        }
        group_sync(gw, my_group);
        for (int c0 = r0 + w_in_group * 32; c0 < r1; c0 += gw * 32) {
            const int k = c0 + lane;
            uint4 a = make_uint4(0, 0, 0, 0), b = make_uint4(0, 0xFFFFFFFFu, kNeverProto, 0xFFFFFFFFu);
            if (k < r1) {
                a = __ldg(&p.clamp[k].a);
                b = __ldg(&p.clamp[k].b);
            }
            // Packets already decided by an earlier (or this) chunk are skipped. The
            // pending set is taken by ballot so that the loop stays warp-uniform;
            // a stale read only costs a redundant check (atomicMin keeps the minimum).
            bool pending = false;
            for (int t0 = 0; t0 < G; t0 += 32) {
                unsigned pend = __ballot_sync(0xFFFFFFFFu, *reinterpret_cast<volatile int *>(&best[t0 + lane]) > c0);
                pending |= pend != 0u;
                // up to four pending packets per pass: four independent test chains and
                // ballots in flight instead of one load-test-vote chain at a time
                while (pend != 0u) {
                    int t[4];
                    bool has[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        has[j] = pend != 0u;
                        t[j] = has[j] ? t0 + __ffs(pend) - 1 : t0;
                        pend &= pend - 1u;  // no-op once empty
                    }
                    unsigned bal[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const Pkt pk = stage[t[j]];
                        bal[j] = __ballot_sync(0xFFFFFFFFu, has[j] && mismatch_clamp(pk, a, b) == 0u);
                    }
                    if (lane == 0) {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (bal[j] != 0u) atomicMin(&best[t[j]], c0 + __ffs(bal[j]) - 1);
                    }
                }
            }
            if (!pending) break;
        }
        group_sync(gw, my_group);
        for (int t = gt; t < G; t += gthreads) {
            const int64_t i = base + t;
            if (i >= p.n) break;
            const int bt = best[t];
            if (p.partial != nullptr) {
                if (bt != INT_MAX) atomicMin(&p.partial[i], bt);
            } else {
                const int r = bt == INT_MAX ? -1 : bt;
                p.out_idx[i] = r;
                p.out_act[i] = r >= 0 ? __ldg(p.action + r) : (uint8_t)FW_DROP;
            }
        }
        group_sync(gw, my_group);
    }
}

__global__ void k_rule_split_finalize(const int32_t *__restrict__ partial, const uint8_t *__restrict__ action,
                                      int64_t n, int32_t *__restrict__ out_idx, uint8_t *__restrict__ out_act) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int v = partial[i];
        const int r = v == kNoMatch ? -1 : v;
        out_idx[i] = r;
        out_act[i] = r >= 0 ? __ldg(action + r) : (uint8_t)FW_DROP;
    }
}


// ------------------------------------------------------------ partitioned kernel (arithmetic records)
struct PartSplitParams {
    const RecArith *rec;      // the class sub-lists, one after another
    const uint32_t *wtop;
    const uint32_t *verdict;  // per record: original index | action << 31
    const int32_t *orig;      // per record: original index
    const uint8_t *class_of;  // protocol -> protocol class
    int32_t n_classes, key_field, key_bits;
    int32_t class_off[kMaxClasses];
    int32_t class_len[kMaxClasses];
    int32_t slices;           // grid mode: slice s takes the chunks k of every class with k % slices == s
    uint32_t one;
    HdrPtrs h;
    int64_t n;
    int32_t *out_idx;
    uint8_t *out_act;
    int32_t *partial;         // grid mode: per-packet minimum original index (pre-set to kNoMatch)
};

constexpr int kWarpGroup = 64;  // packets per warp group (warp and grid mode): two per lane

// Lane's record of chunk k of a class (position 32k + lane of its sub-list), and whether it exists.
__device__ __forceinline__ bool chunk_record(const PartSplitParams &p, int off, int len, int k, int lane,
                                             uint4 &a, uint4 &b, uint32_t &w) {
    const int pos = 32 * k + lane;
    if (pos >= len) return false;
    a = __ldg(&p.rec[off + pos].a);
    b = __ldg(&p.rec[off + pos].b);
    w = __ldg(p.wtop + off + pos);
    return true;
}

// Test the packets of `pend` (bits into the staged group `stage`) against the warp's chunk, up to
// four at a time (independent broadcast loads, tests and votes in flight); report each packet
// whose chunk holds a match through hit(t, position of the first matching record in the chunk).
template <class Hit>
__device__ __forceinline__ void test_pending(uint64_t pend, const PktA *stage, bool vr, const uint4 &a,
                                             const uint4 &b, uint32_t w, uint32_t one, Hit hit) {
    while (pend != 0ull) {
        int t[4];
        bool has[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            has[j] = pend != 0ull;
            t[j] = has[j] ? __ffsll((long long)pend) - 1 : 0;
            pend &= pend - 1ull;  // no-op once empty
        }
        unsigned bal[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const PktA pk = stage[t[j]];
            bal[j] = __ballot_sync(0xFFFFFFFFu, has[j] && vr && !mismatch_arith(pk, a, b, w, one));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (bal[j] != 0u) hit(t[j], __ffs(bal[j]) - 1);
    }
}

// Warp mode (GRID = false): a warp owns a group of 64 packets and walks, class by class, the
// chunks of the class sub-list in order; a packet leaves the pending set at its first match, so
// later chunks skip it. Grid mode (GRID = true): the same per slice (blockIdx.y), which takes
// every slices-th chunk of each class; before a chunk, packets whose running minimum (the
// scratch, from any slice) already lies before the chunk's first rule are dropped, and a match
// is combined into the scratch by atomicMin.
template <bool GRID>
__global__ void __launch_bounds__(256) k_rule_split_part(PartSplitParams p) {
    __shared__ PktA stage_all[8][kWarpGroup];
    __shared__ int best_all[8][kWarpGroup];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    PktA *stage = stage_all[warp];
    int *best = best_all[warp];
    const int nwarps = blockDim.x >> 5;
    const int64_t n_groups = (p.n + kWarpGroup - 1) / kWarpGroup;
    const int slice = GRID ? (int)blockIdx.y : 0, step = GRID ? p.slices : 1;
    for (int64_t g = (int64_t)blockIdx.x * nwarps + warp; g < n_groups; g += (int64_t)gridDim.x * nwarps) {
        const int64_t base = g * kWarpGroup;
        uint32_t cls[2];
        bool valid[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t i = base + lane + 32 * u;
            valid[u] = i < p.n;
            uint32_t s = 0, d = 0, sp = 0, dp = 0, pr = 0;
            if (valid[u]) {
                s = p.h.src[i];
                d = p.h.dst[i];
                sp = p.h.sport[i];
                dp = p.h.dport[i];
                pr = p.h.proto[i];
            }
            stage[lane + 32 * u] = PktA{s, d, sp, x_of(pr, dp)};
            best[lane + 32 * u] = INT_MAX;
            cls[u] = part_class(__ldg(p.class_of + pr), p.key_field, p.key_bits, s, d);
        }
        __syncwarp();
        for (int c = 0; c < p.n_classes; ++c) {
            uint64_t mem = (uint64_t)__ballot_sync(0xFFFFFFFFu, valid[0] && cls[0] == (uint32_t)c) |
                           ((uint64_t)__ballot_sync(0xFFFFFFFFu, valid[1] && cls[1] == (uint32_t)c) << 32);
            const int off = p.class_off[c], len = p.class_len[c];
            const int nck = (len + 31) / 32;
            for (int k = slice; k < nck && mem != 0ull; k += step) {
                uint4 a = make_uint4(0, 0, 0, 0), b = make_uint4(0, 0, 0, 0);
                uint32_t w = 0;
                const bool vr = chunk_record(p, off, len, k, lane, a, b, w);
                if (GRID) {
                    // exact early-out: a packet whose minimum so far precedes this chunk is decided
                    const int first = __ldg(p.orig + off + 32 * k);
                    uint64_t done = 0ull;
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int64_t i = base + lane + 32 * u;
                        const bool before = valid[u] && *reinterpret_cast<volatile int32_t *>(p.partial + i) < first;
                        done |= (uint64_t)__ballot_sync(0xFFFFFFFFu, before) << (32 * u);
                    }
                    mem &= ~done;
                }
                uint64_t hit_mask = 0ull;
                test_pending(mem, stage, vr, a, b, w, p.one, [&](int t, int r) {
                    if (lane == 0) best[t] = 32 * k + r;
                    hit_mask |= 1ull << t;
                });
                mem &= ~hit_mask;  // decided at this chunk: later chunks cannot come first
            }
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t i = base + lane + 32 * u;
            if (!valid[u]) continue;
            const int r = best[lane + 32 * u];
            const int off = p.class_off[cls[u]];
            if (GRID) {
                if (r != INT_MAX) atomicMin(&p.partial[i], __ldg(p.orig + off + r));
            } else {
                const uint32_t vw = r != INT_MAX ? __ldg(p.verdict + off + r) : 0xFFFFFFFFu;
                p.out_idx[i] = r != INT_MAX ? (int32_t)(vw & 0x7FFFFFFFu) : -1;
                p.out_act[i] = r != INT_MAX ? (uint8_t)(vw >> 31) : (uint8_t)FW_DROP;
            }
        }
        __syncwarp();
    }
}

// Warp mode for short sub-lists: k packets x 32/k rules per warp step. The warp's lanes form
// 32 / SEG segments of SEG lanes; each segment works on one packet of the group at a time, lane
// j of the segment testing record k + j of the packet's class sub-list, and the segment's bits of
// the warp vote give that packet's first match among those SEG records (the segment-level
// minimum). A segment whose packet is decided (or whose sub-list ends) takes the next packet of
// the group, so the warp's lanes stay busy across packets of different depths and classes.
template <int SEG>
__global__ void __launch_bounds__(256) k_rule_split_seg(PartSplitParams p) {
    __shared__ PktA stage_all[8][kWarpGroup];
    __shared__ uint8_t cls_all[8][kWarpGroup];
    __shared__ int res_all[8][kWarpGroup];
    constexpr int NS = 32 / SEG;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    PktA *stage = stage_all[warp];
    uint8_t *scls = cls_all[warp];
    int *res = res_all[warp];
    const int seg = lane / SEG, sl = lane % SEG;
    const unsigned seg_mask = (SEG == 32 ? 0xFFFFFFFFu : ((1u << SEG) - 1u)) << (seg * SEG);
    const int nwarps = blockDim.x >> 5;
    const int64_t n_groups = (p.n + kWarpGroup - 1) / kWarpGroup;
    for (int64_t g = (int64_t)blockIdx.x * nwarps + warp; g < n_groups; g += (int64_t)gridDim.x * nwarps) {
        const int64_t base = g * kWarpGroup;
        const int cnt = (int)min((int64_t)kWarpGroup, p.n - base);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int t = lane + 32 * u;
            const int64_t i = base + t;
            uint32_t s = 0, d = 0, sp = 0, dp = 0, pr = 0;
            if (t < cnt) {
                s = p.h.src[i];
                d = p.h.dst[i];
                sp = p.h.sport[i];
                dp = p.h.dport[i];
                pr = p.h.proto[i];
            }
            stage[t] = PktA{s, d, sp, x_of(pr, dp)};
            scls[t] = (uint8_t)part_class(__ldg(p.class_of + pr), p.key_field, p.key_bits, s, d);
        }
        __syncwarp();
        // the segment's current packet, its class's first record and sub-list length, in registers
        int cur = seg, k = 0, next = NS, off = 0, len = 0;
        PktA pk{0, 0, 0, 0};
        auto take = [&]() {
            if (cur < cnt) {
                pk = stage[cur];
                const int c = scls[cur];
                off = p.class_off[c];
                len = p.class_len[c];
            }
        };
        take();
        while (true) {
            const bool active = cur < cnt;
            if (__ballot_sync(0xFFFFFFFFu, active) == 0u) break;
            const int pos = k + sl;
            bool m = false;
            if (active && pos < len) {
                const uint4 a = __ldg(&p.rec[off + pos].a), b = __ldg(&p.rec[off + pos].b);
                m = !mismatch_arith(pk, a, b, __ldg(p.wtop + off + pos), p.one);
            }
            const unsigned bits = __ballot_sync(0xFFFFFFFFu, m) & seg_mask;
            const bool done = active && (bits != 0u || k + SEG >= len);
            if (done && sl == 0) res[cur] = bits != 0u ? k + (__ffs(bits) - 1 - seg * SEG) : INT_MAX;
            // decided segments take the next packets of the group, in segment order
            const unsigned dn = __ballot_sync(0xFFFFFFFFu, done && sl == 0);
            if (done) {
                cur = next + __popc(dn & ((1u << (seg * SEG)) - 1u));
                k = 0;
                take();
            } else {
                k += SEG;
            }
            next += __popc(dn);
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int t = lane + 32 * u;
            if (t >= cnt) continue;
            const int r = res[t];
            const uint32_t vw = r != INT_MAX ? __ldg(p.verdict + p.class_off[scls[t]] + r) : 0xFFFFFFFFu;
            p.out_idx[base + t] = r != INT_MAX ? (int32_t)(vw & 0x7FFFFFFFu) : -1;
            p.out_act[base + t] = r != INT_MAX ? (uint8_t)(vw >> 31) : (uint8_t)FW_DROP;
        }
        __syncwarp();
    }
}

// Block mode (the paper's hybrid, Sec. IV.C): the block's warps share a group of 32 packets per
// warp and split the (class, chunk) work items of that group round-robin; each item tests the
// class's packets not yet decided at an earlier chunk and combines matches by shared atomicMin.
__global__ void __launch_bounds__(512) k_rule_split_part_block(PartSplitParams p) {
    __shared__ PktA stage[512];
    __shared__ int best[512];
    __shared__ uint32_t mem[kMaxClasses][16];  // class membership, one word per 32 packets
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int G = blockDim.x;
    int n_items = 0;
    for (int c = 0; c < p.n_classes; ++c) n_items += (p.class_len[c] + 31) / 32;
    const int64_t n_groups = (p.n + G - 1) / G;
    for (int64_t g = blockIdx.x; g < n_groups; g += gridDim.x) {
        const int64_t i = g * G + threadIdx.x;
        const bool valid = i < p.n;
        uint32_t s = 0, d = 0, sp = 0, dp = 0, pr = 0;
        if (valid) {
            s = p.h.src[i];
            d = p.h.dst[i];
            sp = p.h.sport[i];
            dp = p.h.dport[i];
            pr = p.h.proto[i];
        }
        stage[threadIdx.x] = PktA{s, d, sp, x_of(pr, dp)};
        best[threadIdx.x] = INT_MAX;
        const uint32_t cls = part_class(__ldg(p.class_of + pr), p.key_field, p.key_bits, s, d);
        for (int c = 0; c < p.n_classes; ++c) {
            const unsigned m = __ballot_sync(0xFFFFFFFFu, valid && cls == (uint32_t)c);
            if (lane == 0) mem[c][warp] = m;
        }
        __syncthreads();
        for (int it = warp; it < n_items; it += nwarps) {
            int c = 0, k = it;
            while (k >= (p.class_len[c] + 31) / 32) k -= (p.class_len[c++] + 31) / 32;
            const int off = p.class_off[c], len = p.class_len[c];
            uint4 a = make_uint4(0, 0, 0, 0), b = make_uint4(0, 0, 0, 0);
            uint32_t w = 0;
            const bool vr = chunk_record(p, off, len, k, lane, a, b, w);
            for (int ww = 0; ww < nwarps; ++ww) {
                const uint32_t m = mem[c][ww];
                if (m == 0u) continue;
                // still pending: no match found yet at or before this chunk's first record
                const unsigned pend = m & __ballot_sync(0xFFFFFFFFu, *reinterpret_cast<volatile int *>(&best[32 * ww + lane]) > 32 * k);
                test_pending(pend, stage + 32 * ww, vr, a, b, w, p.one, [&](int t, int r) {
                    if (lane == 0) atomicMin(&best[32 * ww + t], 32 * k + r);
                });
            }
        }
        __syncthreads();
        if (valid) {
            const int r = best[threadIdx.x];
            const uint32_t vw = r != INT_MAX ? __ldg(p.verdict + p.class_off[cls] + r) : 0xFFFFFFFFu;
            p.out_idx[i] = r != INT_MAX ? (int32_t)(vw & 0x7FFFFFFFu) : -1;
            p.out_act[i] = r != INT_MAX ? (uint8_t)(vw >> 31) : (uint8_t)FW_DROP;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ host side
template <class K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// One rule-split classification: warp, block or grid mode (cfg.mode), over the partition
// (default) or the whole list (cfg.partition == 2). Grid mode combines through per-packet
// scratch: `scratch` (n int32 of device memory owned by the caller) when given, else a
// stream-ordered allocation freed on the same stream.
int rule_split_run(const fw_ruleset *rs, const HdrPtrs &h, int64_t n, int32_t *out_idx, uint8_t *out_act,
                   cudaStream_t st, const fw_config &cfg, int32_t *scratch) {
    const bool block_mode = cfg.mode == FW_MODE_RULE_SPLIT_BLOCK;
    const bool grid_mode = cfg.mode == FW_MODE_RULE_SPLIT_GRID;
    if (cfg.partition < 0 || cfg.partition > 2) return FW_EINVAL;
    // Block mode over the partition splits (class, chunk) items among the warps of a packet group;
    // on lists of at most 2,048 reachable rules its per-item overhead outweighs the shorter scans
    // (10K x 16M, 69 reachable rules: 3.12 ms against 1.59 ms for the whole list), so block mode
    // takes the whole list there unless the partition is asked for.
    const bool part = cfg.partition == 1 || (cfg.partition == 0 && !(block_mode && rs->n_eff <= 2048));
    const int per_sm = cfg.blocks_per_sm > 0 ? cfg.blocks_per_sm : 4;
    if (per_sm > 64) return FW_EINVAL;
    cudaError_t e = cudaSuccess;
    int32_t *partial = nullptr;
    auto grid_scratch = [&]() -> cudaError_t {
        if (!grid_mode) return cudaSuccess;
        partial = scratch;
        if (partial == nullptr) {
            cudaError_t a = cudaMallocAsync(reinterpret_cast<void **>(&partial), (size_t)n * sizeof(int32_t), st);
            if (a != cudaSuccess) return a;
        }
        return cudaMemsetAsync(partial, 0x7F, (size_t)n * sizeof(int32_t), st);
    };
    if (part) {
        PartSplitParams p;
        std::memset(&p, 0, sizeof(p));
        p.rec = rs->d_part;
        p.wtop = rs->d_part_wtop;
        p.verdict = rs->d_part_verdict;
        p.orig = rs->d_part_orig;
        p.class_of = rs->d_class_of;
        p.n_classes = rs->n_classes;
        p.key_field = rs->key_field;
        p.key_bits = rs->key_bits;
        int max_chunks = 1;
        for (int c = 0; c < kMaxClasses; ++c) {
            p.class_off[c] = rs->class_off[c];
            p.class_len[c] = rs->class_len[c];
            max_chunks = std::max(max_chunks, (rs->class_len[c] + 31) / 32);
        }
        p.one = 1u;
        p.h = h;
        p.n = n;
        p.out_idx = out_idx;
        p.out_act = out_act;
        if (cfg.packets_per_group != 0) return FW_EINVAL;  // fixed: 64 per warp, 32 per warp in block mode
        const int threads = cfg.block_threads > 0 ? cfg.block_threads : (block_mode ? 512 : 256);
        if (threads % 32 != 0 || threads > (block_mode ? 512 : 256)) return FW_EINVAL;
        // grid mode: no more slices than the longest sub-list has chunks
        p.slices = grid_mode ? std::max(1, std::min(cfg.rule_slices > 0 ? cfg.rule_slices : 8, max_chunks)) : 1;
        if (p.slices > 65535) return FW_EINVAL;
        // warp mode over short sub-lists: 32 / SEG packets of SEG records per warp step
        // (k_rule_split_seg); SEG = segment_rules (2, 4, 8 or 16), default 4 (10K x 16M:
        // 28.1 Gpackets/s at 4, 22.5 at 8, 18.1 at 16)
        const int seg_lanes = cfg.segment_rules > 0 ? cfg.segment_rules : 4;
        if (seg_lanes != 2 && seg_lanes != 4 && seg_lanes != 8 && seg_lanes != 16) return FW_EINVAL;
        const bool seg = !block_mode && !grid_mode && max_chunks <= 2;
        const int G = block_mode ? threads : kWarpGroup * (threads / 32);
        const int64_t groups = (n + G - 1) / G;
        int64_t bx = std::max<int64_t>(1, (int64_t)sm_count(rs->device) * per_sm / p.slices);
        bx = std::max<int64_t>(1, std::min<int64_t>(bx, groups));
        e = grid_scratch();
        p.partial = partial;
        if (e == cudaSuccess) {
            if (block_mode) k_rule_split_part_block<<<(unsigned)bx, threads, 0, st>>>(p);
            else if (grid_mode) k_rule_split_part<true><<<dim3((unsigned)bx, (unsigned)p.slices), threads, 0, st>>>(p);
            else if (seg && seg_lanes == 2) k_rule_split_seg<2><<<(unsigned)bx, threads, 0, st>>>(p);
            else if (seg && seg_lanes == 4) k_rule_split_seg<4><<<(unsigned)bx, threads, 0, st>>>(p);
            else if (seg && seg_lanes == 16) k_rule_split_seg<16><<<(unsigned)bx, threads, 0, st>>>(p);
            else if (seg) k_rule_split_seg<8><<<(unsigned)bx, threads, 0, st>>>(p);
            else k_rule_split_part<false><<<(unsigned)bx, threads, 0, st>>>(p);
            e = cudaGetLastError();
        }
    } else {
        SplitParams p;
        p.clamp = rs->d_clamp;
        p.action = rs->d_action;
        p.n_scan = (int)((rs->n_eff + 3) / 4 * 4);
        p.h = h;
        p.n = n;
        p.out_idx = out_idx;
        p.out_act = out_act;
        p.partial = nullptr;
        const int threads = cfg.block_threads > 0 ? cfg.block_threads : (block_mode ? 512 : 256);
        if (threads % 32 != 0 || threads > 512) return FW_EINVAL;
        int G = cfg.packets_per_group > 0 ? cfg.packets_per_group : (block_mode ? 256 : 64);
        if (G % 32 != 0 || G > 4096) return FW_EINVAL;
        p.group = G;
        const int nwarps = threads / 32;
        // block mode: as many warps per group as the list has 32-rule chunks, up to the block
        p.gw = block_mode ? std::max(1, std::min(nwarps, (p.n_scan + 31) / 32)) : 1;
        const int groups_per_block = nwarps / p.gw;
        const size_t smem = (size_t)groups_per_block * G * (sizeof(Pkt) + sizeof(int));
        if (smem > 227 * 1024) return FW_EINVAL;
        int slices = 1;
        if (grid_mode) {
            slices = cfg.rule_slices > 0 ? cfg.rule_slices : 8;
            slices = std::max(1, std::min(std::min(slices, 65535), (p.n_scan + 31) / 32));
        }
        p.slice_rules = std::max(32, ((p.n_scan + slices - 1) / slices + 31) / 32 * 32);
        slices = std::max(1, (p.n_scan + p.slice_rules - 1) / p.slice_rules);
        const int64_t n_groups = (n + G - 1) / G;
        int64_t bx = std::max<int64_t>(1, (int64_t)sm_count(rs->device) * per_sm / slices);
        bx = std::max<int64_t>(1, std::min<int64_t>(bx, (n_groups + groups_per_block - 1) / groups_per_block));
        e = grid_scratch();
        p.partial = partial;
        if (e == cudaSuccess) {
            if (block_mode) {
                e = allow_smem(k_rule_split<true>, smem);
                if (e == cudaSuccess) k_rule_split<true><<<dim3((unsigned)bx, (unsigned)slices), threads, smem, st>>>(p);
            } else {
                e = allow_smem(k_rule_split<false>, smem);
                if (e == cudaSuccess) k_rule_split<false><<<dim3((unsigned)bx, (unsigned)slices), threads, smem, st>>>(p);
            }
            if (e == cudaSuccess) e = cudaGetLastError();
        }
    }
    if (grid_mode) {
        if (e == cudaSuccess && partial != nullptr) {
            const int fb = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count(rs->device) * 8);
            k_rule_split_finalize<<<std::max(fb, 1), 256, 0, st>>>(partial, rs->d_action, n, out_idx, out_act);
            e = cudaGetLastError();
        }
        if (scratch == nullptr && partial != nullptr) cudaFreeAsync(partial, st);
    }
    return cuda_status(e);
}

int launch_rule_split(const fw_ruleset *rs, const HdrPtrs &h, int64_t n, int32_t *out_idx, uint8_t *out_act,
                      cudaStream_t st, const fw_config &cfg) {
    return rule_split_run(rs, h, n, out_idx, out_act, st, cfg, nullptr);
}

}  // namespace fwk

using namespace fwk;

// ------------------------------------------------------------ allocation-free grid rule split
// Scratch for fw_classify_rule_split_noalloc: the per-packet partial minima of
// the grid rule split, at a fixed address on every device that loads this
// library. Host code must not use the symbol itself as a device address; the
// address is looked up per device with cudaGetSymbolAddress.
static __device__ __align__(256) int32_t g_noalloc_partial[FW_NOALLOC_MAX_PACKETS];

static std::mutex g_noalloc_mu;
static int32_t *g_noalloc_ptr[64] = {};

// Device address of g_noalloc_partial on the current device (looked up once per device).
static int noalloc_scratch(int32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= 64) return FW_EINVAL;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_partial);
        if (e != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return e != cudaSuccess ? cuda_status(e) : FW_ECUDA;
        }
        g_noalloc_ptr[dev] = static_cast<int32_t *>(ptr);
    }
    *out = g_noalloc_ptr[dev];
    return FW_OK;
}

extern "C" int fw_classify_rule_split_noalloc(const fw_ruleset *rs, const fw_headers *hdrs, int64_t n,
                                              int32_t *out_idx, uint8_t *out_act, void *stream,
                                              const fw_config *cfg_in) {
    if (rs == nullptr || n < 0) return set_status(FW_EINVAL);
    if (n > FW_NOALLOC_MAX_PACKETS) return set_status(FW_ERANGE);
    if (n == 0) return set_status(FW_OK);
    if (hdrs == nullptr || hdrs->src == nullptr || hdrs->dst == nullptr || hdrs->sport == nullptr ||
        hdrs->dport == nullptr || hdrs->proto == nullptr || out_idx == nullptr || out_act == nullptr)
        return set_status(FW_EINVAL);
    fw_config cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    if (cfg_in != nullptr) cfg = *cfg_in;
    for (int i = 0; i < 4; ++i)
        if (cfg.reserved[i] != 0) return set_status(FW_EINVAL);
    if (cfg.mode != FW_MODE_AUTO && cfg.mode != FW_MODE_RULE_SPLIT_GRID) return set_status(FW_EINVAL);
    cfg.mode = FW_MODE_RULE_SPLIT_GRID;
    int s = check_device(rs);
    if (s != FW_OK) return set_status(s);
    int32_t *partial = nullptr;
    s = noalloc_scratch(&partial);
    if (s != FW_OK) return set_status(s);
    const HdrPtrs h{hdrs->src, hdrs->dst, hdrs->sport, hdrs->dport, hdrs->proto};
    return set_status(rule_split_run(rs, h, n, out_idx, out_act, reinterpret_cast<cudaStream_t>(stream), cfg,
                                     partial));
}
