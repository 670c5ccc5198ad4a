// Work-list types and the per-item filter routine of the batched persistent
// kernel (fw_batch.cu), shared with the serving scheduler (fw_serve.cu) and the
// device request queue (fw_dqueue.cu).
#pragma once

#include "fw_filter.cuh"

namespace fwk {

// One job of a batched launch: its rule set's partition (protocol classes and
// address key; the concatenated sub-lists in the arithmetic form), its headers
// and outputs.
struct BatchJobDev {
    const RecArith *rec;
    const uint32_t *wtop;
    const uint8_t *action;
    const int32_t *orig;
    const uint32_t *verdict;  // original index | action << 31 per stored record
    const uint8_t *class_of;
    int32_t n_classes;
    int32_t key_field, key_bits;  // address key of the partition (see part_class)
    int32_t vec;  // 1 when the job's buffers allow the vector loads
    int32_t class_off[kMaxClasses];
    int32_t class_len[kMaxClasses];
    HdrPtrs h;
    int64_t n;
    int32_t *out_idx;
    uint8_t *out_act;
    // the rule set's bucket filter (null when it has none): its items are classified through it
    const unsigned char *filter;
    FilterView fv;
    int32_t item_packets;  // packets per work item of this job
    int32_t seg0;          // first rule segment of its scan
};

// One job of a filter-only launch (every job's rule set has a bucket filter): its buffers and its
// rule set's entry in the launch's set table.
struct BatchFilterJob {
    HdrPtrs h;
    int32_t *out_idx;
    uint8_t *out_act;
    int64_t n;
    int32_t set;           // index into the launch's BatchFilterSet table
    int32_t item_packets;  // packets per work item of this job
    int32_t vec;           // 1 when the job's buffers allow the vector loads
    int32_t pad;
};

// A rule set of a filter-only launch: its bucket filter block.
struct BatchFilterSet {
    const unsigned char *filter;
    FilterView fv;
};

// One work item: a run of up to item_packets packets of one job. Items are not stored: job j
// owns items [prefix[j], prefix[j+1]) of the launch (the exclusive prefix of its item counts),
// and a warp that claims item `it` finds its job by a search of the prefix.
struct BatchItem {
    int64_t start;
    int32_t job;
    int32_t count;
};

struct BatchParams {
    const BatchJobDev *jobs;          // the general kernel's jobs
    const BatchFilterJob *fjobs;      // the filter-only kernel's jobs ...
    const BatchFilterSet *fsets;      // ... and their rule sets
    const int64_t *prefix;     // n_jobs + 1 entries: first item of each job, then the item total
    int32_t n_jobs;
    int64_t n_items;
    unsigned long long *next;  // item counter, zeroed before each launch
    int32_t qcap;              // queue capacity per warp (packets)
    uint32_t one;
};

// Packets one item may carry with a queue of `qcap` entries per warp: the
// two-packet scan pads every protocol class region to an even count, at most
// one pad for each of up to kMaxClasses classes.
inline int32_t item_packets(int32_t qcap) { return qcap - kMaxClasses; }

// 1 when a job's header arrays are aligned for the 16-byte vector loads of its scan.
int32_t job_vector_loads(const fw_headers &h);

// Fill a job entry from a rule set and device-accessible buffers (item size and first segment
// of its work items included).
void fill_batch_job(BatchJobDev &d, const fw_ruleset *rs, const fw_headers &h, int64_t n, int32_t *out_idx,
                    uint8_t *out_act, int32_t item_packets, int32_t seg0);

// A rule set's entry of a filter-only launch.
BatchFilterSet batch_filter_set(const fw_ruleset *rs);

// Packets a lane of the batched filter path takes at a time. Two: on four rule sets of 1K..100K
// rules (rows of 1..5 words) one launch over 37.7M packets ran at 82 Gpackets/s, against 77 with
// one packet and 76 with four (whose state no longer fits the 64 registers of two blocks an SM).
constexpr int kBatchFilterPackets = 2;

// Header loads of batch_filter_run: streaming through L1 (default), or from L2 only (HDR_L2:
// for a kernel that outlives the writes of its input buffers and reads them without an acquire
// that would drop stale L1 lines).
template <bool HDR_L2, class T>
__device__ __forceinline__ T batch_hdr_load(const T *p) {
    if constexpr (HDR_L2) return __ldcg(p);
    else return __ldcs(p);
}

// One item of a job with a bucket filter, its block read through L1: P consecutive packets per
// lane (item starts are multiples of four packets, so aligned arrays allow vector loads and
// stores); the classes and first row words of a lane's packets are loaded together, then each
// packet is resolved in turn (filter_packets_wide).
template <int P, bool HDR_L2 = false>
__device__ __forceinline__ void batch_filter_run(const BatchFilterJob &J, const BatchFilterSet &S,
                                                 const BatchItem &item, int lane, uint32_t one) {
    static_assert(P == 1 || P == 2, "one or two packets a lane");
    const FilterView fv = S.fv;
    const unsigned char *__restrict__ base = S.filter;
    const int64_t st = item.start;
    const bool vin = J.vec != 0;
    const bool vout = vin && (reinterpret_cast<uintptr_t>(J.out_idx + st) % (4 * P) == 0) &&
                      (reinterpret_cast<uintptr_t>(J.out_act + st) % P == 0);
    for (int q = P * lane; q < item.count; q += 32 * P) {
        const int64_t i = st + q;
        const int m = min(P, item.count - q);
        uint32_t s[P], d[P], sp[P], dp[P], pr[P], vw[P];
        if (P == 2 && vin && m == P) {
            const uint2 a = batch_hdr_load<HDR_L2>(reinterpret_cast<const uint2 *>(J.h.src + i));
            const uint2 b = batch_hdr_load<HDR_L2>(reinterpret_cast<const uint2 *>(J.h.dst + i));
            const uint32_t c = batch_hdr_load<HDR_L2>(reinterpret_cast<const unsigned int *>(J.h.sport + i));
            const uint32_t e = batch_hdr_load<HDR_L2>(reinterpret_cast<const unsigned int *>(J.h.dport + i));
            const uint32_t f = batch_hdr_load<HDR_L2>(reinterpret_cast<const unsigned short *>(J.h.proto + i));
            s[0] = a.x; s[P - 1] = a.y;
            d[0] = b.x; d[P - 1] = b.y;
            sp[0] = c & 0xFFFFu; sp[P - 1] = c >> 16;
            dp[0] = e & 0xFFFFu; dp[P - 1] = e >> 16;
            pr[0] = f & 0xFFu; pr[P - 1] = f >> 8;
        } else {
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const int64_t ik = k < m ? i + k : i;  // past the item's end: a copy of its first packet
                if constexpr (HDR_L2) {
                    s[k] = __ldcg(J.h.src + ik);
                    d[k] = __ldcg(J.h.dst + ik);
                    sp[k] = __ldcg(reinterpret_cast<const unsigned short *>(J.h.sport + ik));
                    dp[k] = __ldcg(reinterpret_cast<const unsigned short *>(J.h.dport + ik));
                    pr[k] = __ldcg(reinterpret_cast<const unsigned char *>(J.h.proto + ik));
                } else {
                    s[k] = J.h.src[ik];
                    d[k] = J.h.dst[ik];
                    sp[k] = J.h.sport[ik];
                    dp[k] = J.h.dport[ik];
                    pr[k] = J.h.proto[ik];
                }
            }
        }
        filter_packets_wide<P>(base, fv, s, d, sp, dp, pr, one, vw);
        int32_t oi[P];
        uint32_t oa = 0;
#pragma unroll
        for (int k = 0; k < P; ++k) {
            oi[k] = vw[k] == 0xFFFFFFFFu ? -1 : (int32_t)(vw[k] & 0x7FFFFFFFu);
            oa |= (vw[k] == 0xFFFFFFFFu ? (uint32_t)FW_DROP : (vw[k] >> 31)) << (8 * k);
        }
        if (P == 2 && vout && m == P) {
            __stcs(reinterpret_cast<int2 *>(J.out_idx + i), make_int2(oi[0], oi[P - 1]));
            __stcs(reinterpret_cast<unsigned short *>(J.out_act + i), (unsigned short)oa);
        } else {
#pragma unroll
            for (int k = 0; k < P; ++k)
                if (k < m) {
                    J.out_idx[i + k] = oi[k];
                    J.out_act[i + k] = (uint8_t)(oa >> (8 * k));
                }
        }
    }
}

// Block size and default resident blocks per SM of the filter-only batched kernel.
constexpr int kBatchFilterThreads = 512;
constexpr int kBatchFilterMinBlocks = 2;

// Zero the item counter and launch the persistent kernel on `st` (nothing but
// the counter reset when n_items is 0); d_prefix holds n_jobs + 1 item offsets. The kernel's shared-memory limit must
// have been raised with prepare_batch_kernel for `qcap` and `threads`.
cudaError_t launch_batch(const BatchJobDev *d_jobs, const int64_t *d_prefix, int32_t n_jobs, int64_t n_items,
                         unsigned long long *d_next, int32_t qcap, int threads, int64_t blocks, cudaStream_t st);
// The filter-only kernel (built for filter_minb = 2 or 3 resident blocks per SM) over compact jobs
// and their set table; *d_next must already be zero on `st`.
cudaError_t launch_batch_filter(const BatchFilterJob *d_jobs, const BatchFilterSet *d_sets, const int64_t *d_prefix,
                                int32_t n_jobs, int64_t n_items, unsigned long long *d_next, int64_t blocks,
                                cudaStream_t st, int filter_minb);
cudaError_t prepare_batch_kernel(size_t smem_bytes);
size_t batch_smem_bytes(int threads, int32_t qcap);  // dynamic shared memory of k_batch

}  // namespace fwk
