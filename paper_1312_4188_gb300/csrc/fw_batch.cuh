// Work-list types of the batched persistent kernel (fw_batch.cu), shared with
// the serving scheduler (fw_serve.cu).
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
