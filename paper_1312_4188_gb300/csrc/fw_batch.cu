// Batched classification: many (rule set, packet batch) jobs in one
// persistent launch, optionally replayed from a CUDA graph.
//
// The paper's data-parallel firewall accumulates a set of packets and checks
// them in parallel against one rule set (Sec. IV.A); its conclusions point to
// asynchronous launches to cut per-batch delay (Sec. V). Here a plan splits
// every job into items, runs of up to `packets_per_item` packets. Items are
// not stored: the plan keeps, per job, the offset of its first item (the
// exclusive prefix of the jobs' item counts), and a persistent grid of warps
// claims item indices from a global counter (dynamic scheduling, so cheap and
// expensive items balance) and finds each item's job by a search of that
// prefix. Each warp classifies its item against the item's own rule set, read
// through L1: through the rule set's bucket filter when it has one
// (fw_filter.cuh), else with the two-packets-per-lane first-match scan of
// fw_scan.cuh. Jobs are ordered by decreasing rule-set size so the long scans
// start first. Per size class of rule set (by reachable rules) the plan
// carries its own item size and first rule segment, chosen by the autotuner.
#include <algorithm>
#include <map>
#include <cstring>
#include <vector>

#include "fw_alloc.h"
#include "fw_batch.cuh"

namespace fwk {


// Claim the next item of a launch for the calling warp: its index from the global counter, its
// job by a search of the item prefix (the last j with prefix[j] <= index). False when none is left.
__device__ __forceinline__ bool batch_claim(const BatchParams &p, int lane, int &job, int64_t &it) {
    unsigned long long x = 0;
    if (lane == 0) x = atomicAdd(p.next, 1ull);
    x = __shfl_sync(0xFFFFFFFFu, x, 0);
    if (x >= (unsigned long long)p.n_items) return false;
    int j = 0;
    if (lane == 0) {
        int lo = 0, hi = p.n_jobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(p.prefix + mid) <= (int64_t)x) lo = mid;
            else hi = mid - 1;
        }
        j = lo;
    }
    job = __shfl_sync(0xFFFFFFFFu, j, 0);
    it = (int64_t)x;
    return true;
}

// A filter job's item inside the general kernel (whose jobs carry their rule set's fields). Kept
// out of line so that its registers do not add to the scan path's.
__device__ __noinline__ void batch_filter_item(const BatchJobDev &J, const BatchItem &item, int lane, uint32_t one) {
    BatchFilterJob fj;
    fj.h = J.h;
    fj.out_idx = J.out_idx;
    fj.out_act = J.out_act;
    fj.n = J.n;
    fj.vec = J.vec;
    BatchFilterSet fs;
    fs.filter = J.filter;
    fs.fv = J.fv;
    batch_filter_run<kBatchFilterPackets>(fj, fs, item, lane, one);
}

// The persistent kernel of launches whose jobs all have a bucket filter: compact jobs and a table of
// their rule sets, no scan queue in shared memory, so more warps fit on an SM and the L1 cache
// keeps its whole capacity for the filter blocks. MINB resident blocks per SM: 2 (64 registers a
// thread) or 3 (40).
template <int MINB>
__global__ void __launch_bounds__(kBatchFilterThreads, MINB) k_batch_filter(BatchParams p) {
    const int lane = threadIdx.x & 31;
    int job;
    int64_t it;
    while (batch_claim(p, lane, job, it)) {
        const BatchFilterJob &J = p.fjobs[job];
        BatchItem item;
        item.job = job;
        item.start = (it - __ldg(p.prefix + job)) * J.item_packets;
        item.count = (int32_t)min((int64_t)J.item_packets, J.n - item.start);
        batch_filter_run<kBatchFilterPackets>(J, p.fsets[J.set], item, lane, p.one);
    }
}

__global__ void __launch_bounds__(1024) k_batch(BatchParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    uint4 *Q = reinterpret_cast<uint4 *>(smem) + (size_t)warp * p.qcap;
    int *wc = reinterpret_cast<int *>(smem + (size_t)nw * p.qcap * sizeof(uint4)) + warp * 2 * kMaxClasses;
    int job;
    int64_t it;
    while (batch_claim(p, lane, job, it)) {
        const BatchJobDev &J = p.jobs[job];
        BatchItem item;
        item.job = job;
        item.start = ((int64_t)it - __ldg(p.prefix + job)) * J.item_packets;
        item.count = (int32_t)min((int64_t)J.item_packets, J.n - item.start);
        if (J.filter != nullptr) {
            batch_filter_item(J, item, lane, p.one);
            continue;
        }
        BatchTarget<PolArith> t;
        t.h = J.h;
        t.n = J.n;
        t.gv = PolArith::View{J.rec, J.wtop};
        t.sv = t.gv;
        t.n_smem = 0;  // rules come through L1: jobs of one launch use different rule sets
        t.n_scan = 0;
        t.n_classes = J.n_classes;
        t.key_field = J.key_field;
        t.key_bits = J.key_bits;
        t.class_off = J.class_off;
        t.class_len = J.class_len;
        t.class_of = J.class_of;
        t.orig = J.orig;
        t.verdict = J.verdict;
        t.action = J.action;
        t.out_idx = J.out_idx;
        t.out_act = J.out_act;
        t.seg0 = J.seg0;
        t.one = p.one;
        if (J.vec) run_batch_pairs<PolArith, true>(t, item.start, item.count, Q, wc, lane);
        else run_batch_pairs<PolArith, false>(t, item.start, item.count, Q, wc, lane);
    }
}

static bool al(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int32_t job_vector_loads(const fw_headers &h) {
    return al(h.src, 16) && al(h.dst, 16) && al(h.sport, 8) && al(h.dport, 8) && al(h.proto, 4);
}

void fill_batch_job(BatchJobDev &d, const fw_ruleset *rs, const fw_headers &h, int64_t n, int32_t *out_idx,
                    uint8_t *out_act, int32_t item_packets, int32_t seg0) {
    d.rec = rs->d_part;
    d.wtop = rs->d_part_wtop;
    d.action = rs->d_action;
    d.orig = rs->d_part_orig;
    d.verdict = rs->d_part_verdict;
    d.class_of = rs->d_class_of;
    d.n_classes = rs->n_classes;
    d.key_field = rs->key_field;
    d.key_bits = rs->key_bits;
    for (int c = 0; c < kMaxClasses; ++c) {
        d.class_off[c] = rs->class_off[c];
        d.class_len[c] = rs->class_len[c];
    }
    d.vec = job_vector_loads(h);
    d.h = HdrPtrs{h.src, h.dst, h.sport, h.dport, h.proto};
    d.n = n;
    d.out_idx = out_idx;
    d.out_act = out_act;
    d.filter = rs->filter_words > 0 ? rs->d_filter : nullptr;
    d.fv = filter_view(rs);
    d.item_packets = item_packets;
    d.seg0 = seg0;
}

size_t batch_smem_bytes(int threads, int32_t qcap) {
    return (size_t)(threads / 32) * ((size_t)qcap * sizeof(uint4) + 2 * kMaxClasses * sizeof(int));
}

cudaError_t prepare_batch_kernel(size_t smem_bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    // the filter-only kernel uses no shared memory: give the L1 cache the whole carve-out
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_batch_filter<2>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_batch_filter<3>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    return e;
}

cudaError_t launch_batch(const BatchJobDev *d_jobs, const int64_t *d_prefix, int32_t n_jobs, int64_t n_items,
                         unsigned long long *d_next, int32_t qcap, int threads, int64_t blocks, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d_next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || n_items == 0 || n_jobs == 0) return e;
    BatchParams p{};
    p.jobs = d_jobs;
    p.prefix = d_prefix;
    p.n_jobs = n_jobs;
    p.n_items = n_items;
    p.next = d_next;
    p.qcap = qcap;
    p.one = 1u;
    k_batch<<<(unsigned)blocks, threads, batch_smem_bytes(threads, qcap), st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_batch_filter(const BatchFilterJob *d_jobs, const BatchFilterSet *d_sets, const int64_t *d_prefix,
                                int32_t n_jobs, int64_t n_items, unsigned long long *d_next, int64_t blocks,
                                cudaStream_t st, int filter_minb) {
    if (n_items == 0 || n_jobs == 0) return cudaSuccess;
    BatchParams p{};
    p.fjobs = d_jobs;
    p.fsets = d_sets;
    p.prefix = d_prefix;
    p.n_jobs = n_jobs;
    p.n_items = n_items;
    p.next = d_next;
    p.one = 1u;
    if (filter_minb == 3) k_batch_filter<3><<<(unsigned)blocks, kBatchFilterThreads, 0, st>>>(p);
    else k_batch_filter<2><<<(unsigned)blocks, kBatchFilterThreads, 0, st>>>(p);
    return cudaGetLastError();
}

BatchFilterSet batch_filter_set(const fw_ruleset *rs) {
    BatchFilterSet s;
    s.filter = rs->filter_words > 0 ? rs->d_filter : nullptr;
    s.fv = filter_view(rs);
    return s;
}

}  // namespace fwk

struct fw_plan {
    int device = 0;
    int threads = 1024;
    int64_t blocks = 1;
    size_t smem = 0;
    int64_t n_items = 0;
    int64_t n_jobs = 0;
    int64_t packets = 0;
    fwk::BatchJobDev *d_jobs = nullptr;       // the general kernel's jobs, or
    fwk::BatchFilterJob *d_fjobs = nullptr;   // the filter-only kernel's jobs
    fwk::BatchFilterSet *d_fsets = nullptr;   // and their rule sets
    int64_t *d_prefix = nullptr;  // n_jobs + 1 item offsets
    unsigned long long *d_next = nullptr;
    int32_t qcap = 256;
    int filter_minb = 0;  // every job has a bucket filter: k_batch_filter<filter_minb> runs (else 0)
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

using namespace fwk;

extern "C" void fw_plan_destroy(fw_plan *pl) {
    if (pl == nullptr) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    cudaFree(pl->d_jobs);
    cudaFree(pl->d_fjobs);
    cudaFree(pl->d_fsets);
    cudaFree(pl->d_prefix);
    cudaFree(pl->d_next);
    delete pl;
}

extern "C" int fw_plan_create(const fw_job *jobs, int64_t n_jobs, const fw_plan_config *cfg_in, fw_plan **out) {
    if (out == nullptr) return set_status(FW_EINVAL);
    *out = nullptr;
    if (n_jobs < 0 || (n_jobs > 0 && jobs == nullptr) || n_jobs > (1 << 24)) return set_status(FW_EINVAL);
    fw_plan_config cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    if (cfg_in) cfg = *cfg_in;
    const int n_classes = cfg.n_classes > 0 ? cfg.n_classes : 1;
    if (n_classes > 4) return set_status(FW_EINVAL);
    int32_t per_item[4], seg0[4];
    int32_t qcap = 0;
    for (int c = 0; c < n_classes; ++c) {
        per_item[c] = cfg.packets_per_item[c] > 0 ? cfg.packets_per_item[c] : 256;
        seg0[c] = cfg.segment_rules[c] > 0 ? cfg.segment_rules[c] : 64;
        if (per_item[c] % 128 != 0 || per_item[c] > 4096 || seg0[c] % 4 != 0) return set_status(FW_EINVAL);
        qcap = std::max(qcap, per_item[c]);
    }
    // default shape: 512-thread blocks, two per SM (256 sets x 31M packets: 2.25 ms against
    // 2.32 ms for one 1,024-thread block per SM); the kernel allows 1,024 threads per SM
    const int threads = cfg.block_threads > 0 ? cfg.block_threads : 512;
    if (threads % 32 != 0 || threads > 1024) return set_status(FW_EINVAL);
    const size_t smem = batch_smem_bytes(threads, qcap);
    if (smem > 227 * 1024) return set_status(FW_EINVAL);

    std::vector<BatchJobDev> hj((size_t)n_jobs);
    int64_t packets = 0;
    // jobs (and so their items) longest scans first
    std::vector<int64_t> order((size_t)n_jobs);
    for (int64_t j = 0; j < n_jobs; ++j) order[j] = j;
    for (int64_t j = 0; j < n_jobs; ++j) {
        const fw_job &J = jobs[j];
        if (J.rs == nullptr || J.n < 0 || J.n > INT32_MAX) return set_status(FW_EINVAL);
        if (J.n > 0 && (!J.hdrs.src || !J.hdrs.dst || !J.hdrs.sport || !J.hdrs.dport || !J.hdrs.proto ||
                        !J.out_rule_idx || !J.out_action))
            return set_status(FW_EINVAL);
    }
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return jobs[a].rs->n_eff > jobs[b].rs->n_eff; });
    // every job through a bucket filter: the filter-only kernel
    bool filter_only = true;
    for (int64_t j = 0; j < n_jobs; ++j)
        if (jobs[j].n > 0 && jobs[j].rs->filter_words == 0) filter_only = false;
    std::vector<int64_t> prefix((size_t)n_jobs + 1, 0);
    // filter-only: compact jobs and a table of their distinct rule sets
    std::vector<BatchFilterJob> hf;
    std::vector<BatchFilterSet> hs;
    std::map<const fw_ruleset *, int32_t> set_index;
    if (filter_only) hf.resize((size_t)n_jobs);
    for (int64_t k = 0; k < n_jobs; ++k) {
        const fw_job &J = jobs[order[k]];
        int c = 0;
        while (c < n_classes - 1 && J.rs->n_eff > cfg.class_max_rules[c]) ++c;
        const int32_t B = item_packets(per_item[c]);
        fill_batch_job(hj[k], J.rs, J.hdrs, J.n, J.out_rule_idx, J.out_action, B, seg0[c]);
        if (filter_only) {
            auto ins = set_index.emplace(J.rs, (int32_t)hs.size());
            if (ins.second) hs.push_back(batch_filter_set(J.rs));
            BatchFilterJob &f = hf[(size_t)k];
            f = BatchFilterJob{};
            f.h = hj[k].h;
            f.out_idx = hj[k].out_idx;
            f.out_act = hj[k].out_act;
            f.n = J.n;
            f.set = ins.first->second;
            f.item_packets = B;
            f.vec = hj[k].vec;
        }
        prefix[k + 1] = prefix[k] + (J.n + B - 1) / B;
        packets += J.n;
    }
    fw_plan *pl = new (std::nothrow) fw_plan();
    if (pl == nullptr) return set_status(FW_ENOMEM);
    cudaGetDevice(&pl->device);
    pl->threads = threads;
    pl->smem = smem;
    pl->qcap = qcap;
    pl->n_items = prefix[(size_t)n_jobs];
    pl->n_jobs = n_jobs;
    pl->packets = packets;
    const int per_sm = cfg.blocks_per_sm > 0 ? cfg.blocks_per_sm : filter_only ? kBatchFilterMinBlocks : 2;
    pl->filter_minb = filter_only ? (per_sm >= 3 ? 3 : 2) : 0;
    const int wpb = (filter_only ? kBatchFilterThreads : threads) / 32;
    pl->blocks = std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count(pl->device) * per_sm, (pl->n_items + wpb - 1) / wpb));
    cudaError_t e = cudaSuccess;
    if (filter_only) {
        e = dev_malloc(&pl->d_fjobs, std::max<size_t>(1, hf.size()) * sizeof(BatchFilterJob));
        if (e == cudaSuccess) e = dev_malloc(&pl->d_fsets, std::max<size_t>(1, hs.size()) * sizeof(BatchFilterSet));
        if (e == cudaSuccess && !hf.empty())
            e = cudaMemcpy(pl->d_fjobs, hf.data(), hf.size() * sizeof(BatchFilterJob), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !hs.empty())
            e = cudaMemcpy(pl->d_fsets, hs.data(), hs.size() * sizeof(BatchFilterSet), cudaMemcpyHostToDevice);
    } else {
        e = dev_malloc(&pl->d_jobs, std::max<size_t>(1, hj.size()) * sizeof(BatchJobDev));
        if (e == cudaSuccess && !hj.empty())
            e = cudaMemcpy(pl->d_jobs, hj.data(), hj.size() * sizeof(BatchJobDev), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = dev_malloc(&pl->d_prefix, prefix.size() * sizeof(int64_t));
    if (e == cudaSuccess) e = dev_malloc(&pl->d_next, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(pl->d_prefix, prefix.data(), prefix.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = prepare_batch_kernel(smem);
    if (e != cudaSuccess) {
        fw_plan_destroy(pl);
        cudaGetLastError();
        return set_status(cuda_status(e));
    }
    *out = pl;
    return FW_OK;
}

static cudaError_t enqueue_plan(fw_plan *pl, cudaStream_t st) {
    if (pl->filter_minb == 0)
        return launch_batch(pl->d_jobs, pl->d_prefix, (int32_t)pl->n_jobs, pl->n_items, pl->d_next, pl->qcap,
                            pl->threads, pl->blocks, st);
    cudaError_t e = cudaMemsetAsync(pl->d_next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    return launch_batch_filter(pl->d_fjobs, pl->d_fsets, pl->d_prefix, (int32_t)pl->n_jobs, pl->n_items, pl->d_next,
                               pl->blocks, st, pl->filter_minb);
}

extern "C" int fw_plan_launch(fw_plan *pl, void *stream) {
    if (pl == nullptr) return set_status(FW_EINVAL);
    return set_status(cuda_status(enqueue_plan(pl, reinterpret_cast<cudaStream_t>(stream))));
}

extern "C" int fw_plan_launch_graph(fw_plan *pl, void *stream) {
    if (pl == nullptr) return set_status(FW_EINVAL);
    cudaError_t e = cudaSuccess;
    if (pl->exec == nullptr) {
        if (pl->cap_stream == nullptr) e = cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t eq = enqueue_plan(pl, pl->cap_stream);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(pl->cap_stream, &g);
            if (eq != cudaSuccess) e = eq;
            if (e == cudaSuccess) {
                pl->graph = g;
                e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
            } else if (g) {
                cudaGraphDestroy(g);
            }
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_status(cuda_status(e));
        }
    }
    return set_status(cuda_status(cudaGraphLaunch(pl->exec, reinterpret_cast<cudaStream_t>(stream))));
}

extern "C" int64_t fw_plan_items(const fw_plan *pl) { return pl ? pl->n_items : -1; }

extern "C" int fw_plan_kernel(const fw_plan *pl) { return pl ? pl->filter_minb : -1; }
